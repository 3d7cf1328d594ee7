"""The no-allocation clutter filter entry point (fq_clutter_svd_noalloc)
against the workspace entry point (fq_clutter_svd) and the FP64 oracle,
through the C ABI.

This serves callers that cannot provide a workspace: the call uses a
scratch array built into the library.  Several calls in a row on
different inputs must each agree with the workspace path and with the
oracle, so nothing left in the shared array from the previous call leaks
into the next result.  The last case sits at the documented limit of 256
frames with enough pixels that the Gram partial sums take the capped
16-chunk layout, and its eigen-solver matrix lives in the array (it does
not fit in shared memory at that size)."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq

pytestmark = pytest.mark.gpu

PD_TOL = 1e-3


def _ensemble(P, F, k, seed):
    """Rank-k clutter with a spectral gap plus white noise, rounded to FP32
    (the input both sides see)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((F, F)) + 1j * rng.standard_normal((F, F)))
    Uc, _ = np.linalg.qr(rng.standard_normal((P, k)) + 1j * rng.standard_normal((P, k)))
    S = (Uc * (1e3 * np.linspace(2.0, 1.0, k))) @ Q[:, :k].conj().T
    S = S + (rng.standard_normal((P, F)) + 1j * rng.standard_normal((P, F))) * 0.3
    S = S.astype(np.complex64).astype(np.complex128)
    return S, torch.from_numpy(np.stack([S.real, S.imag], -1).astype(np.float32)).cuda()


def _rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _h(t):
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def cases():
    fqbuild.build()
    fq.lib()
    # (P, F, k_cut, energy threshold); the last one is the F = 256 limit
    specs = [(4096, 32, 3, 0.9), (3000, 200, -1, 0.9), (1024, 256, 3, 0.9)]
    out = []
    for i, (P, F, k_cut, thr) in enumerate(specs):
        S, Sd = _ensemble(P, F, 3 if k_cut < 0 else k_cut, seed=1 + i)
        out.append((S, Sd, k_cut, thr, oracle.svd_filter(S, k_cut=k_cut, energy_thresh=thr)))
    return out


def test_noalloc_matches_workspace_path_and_oracle(cases):
    for S, Sd, k_cut, thr, (S_f, pd_o, sg, k_o) in cases:
        F = S.shape[1]
        ref = fq.fq_clutter_svd(Sd, k_cut=k_cut, energy_thresh=thr)
        fq.fq_clutter_status(ref["ws"])
        got = fq.fq_clutter_svd_noalloc(Sd, k_cut=k_cut, energy_thresh=thr)
        torch.cuda.synchronize()
        fq.fq_clutter_status(None)  # the array's status word: the eigen-solver converged
        k = int(got["k"].item())
        assert k == int(ref["k"].item()) == k_o
        lam = _h(got["eigvals"])
        # the workspace path
        lam_r = _h(ref["eigvals"])
        assert np.abs(lam - lam_r).max() <= 1e-5 * lam_r[0]
        assert _rel(_h(got["pd"]), _h(ref["pd"])) <= PD_TOL
        assert _rel(_h(got["iq_f"]), _h(ref["iq_f"])) <= PD_TOL
        # the FP64 oracle: eigenvalues = sigma^2 within the FP32 solver's
        # backward error (~F eps ||G||), power Doppler and filtered ensemble
        assert np.abs(lam - sg ** 2).max() <= max(2e-6, 2 * F * 2.0 ** -24) * sg[0] ** 2
        assert _rel(_h(got["pd"]), pd_o) <= PD_TOL
        iq_f = _h(got["iq_f"])
        assert _rel(iq_f[..., 0] + 1j * iq_f[..., 1], S_f) <= PD_TOL


def test_noalloc_rejects_too_many_frames():
    fqbuild.build()
    L = fq.lib()
    st = L.fq_clutter_svd_noalloc(C.c_void_p(256), 0, 100, 300, 2, 0.9, None, None, None, None, None)
    assert st == 2  # FQ_ERR_SHAPE
    assert b"256" in L.fq_last_error()

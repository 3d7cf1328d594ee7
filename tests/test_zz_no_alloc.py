"""The no-allocation clutter filter entry point (fq_clutter_svd_noalloc)
against the workspace entry point (fq_clutter_svd), through the C ABI.

This serves callers that cannot provide a workspace: the call uses a
scratch array built into the library.  Two calls in a row on different
inputs must each agree with the workspace path, so nothing left in the
shared array from the previous call leaks into the next result."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq

pytestmark = pytest.mark.gpu

PD_TOL = 1e-3


def _ensemble(P, F, k, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((F, F)) + 1j * rng.standard_normal((F, F)))
    Uc, _ = np.linalg.qr(rng.standard_normal((P, k)) + 1j * rng.standard_normal((P, k)))
    S = (Uc * (1e3 * np.linspace(2.0, 1.0, k))) @ Q[:, :k].conj().T
    S = S + (rng.standard_normal((P, F)) + 1j * rng.standard_normal((P, F))) * 0.3
    return torch.from_numpy(np.stack([S.real, S.imag], -1).astype(np.float32)).cuda()


def _rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_workspace_path_twice():
    fqbuild.build()
    fq.lib()
    cases = [(_ensemble(4096, 32, 3, 1), 3, 0.9), (_ensemble(3000, 200, 2, 2), -1, 0.9)]
    for S, k_cut, thr in cases:
        ref = fq.fq_clutter_svd(S, k_cut=k_cut, energy_thresh=thr)
        fq.fq_clutter_status(ref["ws"])
        got = fq.fq_clutter_svd_noalloc(S, k_cut=k_cut, energy_thresh=thr)
        torch.cuda.synchronize()
        assert int(got["k"].item()) == int(ref["k"].item())
        lam_r = ref["eigvals"].cpu().numpy()
        assert np.abs(got["eigvals"].cpu().numpy() - lam_r).max() <= 1e-5 * lam_r[0]
        assert _rel(got["pd"], ref["pd"]) <= PD_TOL
        assert _rel(got["iq_f"], ref["iq_f"]) <= PD_TOL


def test_noalloc_rejects_too_many_frames():
    fqbuild.build()
    L = fq.lib()
    st = L.fq_clutter_svd_noalloc(C.c_void_p(256), 0, 100, 300, 2, 0.9, None, None, None, None, None)
    assert st == 2  # FQ_ERR_SHAPE
    assert b"256" in L.fq_last_error()

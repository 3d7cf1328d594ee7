"""The paper's explicit DAS-matrix route (Sec. 2.4.1, Alg. 3) on the GPU:
the matrices against the oracle's, and their product against the direct
DAS of the oracle and of the fused kernel, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_05464_gb300 import fq
from paper_2509_05464_gb300 import workload as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cases():
    c1 = W.config1(n_frames=3)
    c2 = W.shrink(W.config2(n_scat=100_000, n_frames=3), max_scat=2000, grid_div=4)
    return {"c1": c1, "c2": c2}


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_matrices_match_the_oracle(cfg):
    w = _cases()[cfg]
    dm = fq.DasMatrix(w.probe, w.tilt_x, w.tilt_y, w.grid)
    rp_o, col_o, val_o = oracle.das_matrix(w.probe, w.tilt_x, w.tilt_y, w.grid)
    rp = host(dm.row_ptr)
    counts, counts_o = np.diff(rp), np.diff(rp_o)
    # the aperture decision is the same binary32 test on both sides; a
    # sample index (floor of the delay) may differ only when the delay is
    # within rounding of an integer sample
    same = counts == counts_o
    assert same.mean() >= 0.9999
    col, val = host(dm.col)[: dm.nnz], host(dm.val)[: dm.nnz]
    v = val[:, 0] + 1j * val[:, 1]
    rows = np.nonzero(same)[0]
    k = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    ko = np.concatenate([np.arange(rp_o[r], rp_o[r + 1]) for r in rows])
    agree = col[k] == col_o[ko]
    assert agree.mean() >= 0.9999
    assert np.abs(v[k][agree] - val_o[ko][agree]).max() <= 2e-6


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_apply_equals_das(cfg):
    w = _cases()[cfg]
    F = w.n_frames
    pos = np.stack([oracle.advect(w.p0, w.seg, w.flow, *_tables(w), f / w.prf) for f in range(F)])
    rf = np.stack([oracle.simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos[f], w.amp) for f in range(F)]
                  ).astype(np.float32)
    A, M, Ns = len(w.tilt_x), w.probe.nx * w.probe.ny, w.probe.n_samples
    ch = fq.fq_rf2iq(w.probe, A * M, F, dev(rf))
    dm = fq.DasMatrix(w.probe, w.tilt_x, w.tilt_y, w.grid)
    got = host(dm.apply(ch, F))
    fused = host(fq.fq_das(w.probe, w.tilt_x, w.tilt_y, ch, F, w.grid))
    want = oracle.beamform(w.probe, w.tilt_x, w.tilt_y, rf, w.grid)
    g = got[..., 0] + 1j * got[..., 1]
    assert rel_l2(np.stack([g.real, g.imag]), np.stack([want.real, want.imag])) <= 1e-5
    assert rel_l2(got, fused) <= 2e-6


def _tables(w):
    return W.segment_table(w), W.motion_table(w.motion)


def test_frame_limit_and_bf16():
    w = _cases()["c1"]
    dm = fq.DasMatrix(w.probe, w.tilt_x, w.tilt_y, w.grid)
    A, M, Ns = len(w.tilt_x), w.probe.nx * w.probe.ny, w.probe.n_samples
    ch = torch.zeros((A * M, Ns, fq.frame_pad(417), 2), device="cuda")
    with pytest.raises(fq.FqError):
        dm.apply(ch, 417)
    # BF16 channel data: the matrices interpolate the widened values in
    # FP32, so they match the FP32 DAS of the same BF16-rounded data
    ch16 = torch.randn((A * M, Ns, fq.frame_pad(3), 2), device="cuda").bfloat16()
    a = host(dm.apply(ch16, 3))
    b = host(fq.fq_das(w.probe, w.tilt_x, w.tilt_y, ch16.float(), 3, w.grid))
    assert rel_l2(a, b) <= 2e-6

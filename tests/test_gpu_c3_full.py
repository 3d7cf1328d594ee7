"""Checks at the full size of the 3D volumetric workload (32x32 matrix array,
9 plane-wave tilts, 1536 samples, 500k scatterers in a vessel tree, 100
frames, 128^3 voxels), in the launch configuration the benchmark times (RF
and channel IQ stored in BF16, Casorati matrix FP32): sampled outputs the
oracle computes one by one, and properties that hold at any size.  The
whole path against the oracle runs on a seeded subset of the same workload.

Tolerances: RF and IQ relative L2 <= 1e-5 with FP32 storage and <= 1e-2
with BF16 storage; power Doppler <= 1e-3 (FP32 and FP16 storage)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq
from paper_2509_05464_gb300 import workload as W
from paper_2509_05464_gb300.pipeline import Pipeline

pytestmark = pytest.mark.gpu

RF_TOL = 1e-5
BF16_TOL = 1e-2
PD_TOL = 1e-3
BENCH_STORAGE = dict(rf_dtype=torch.bfloat16, ch_dtype=torch.bfloat16, iq_dtype=torch.float32)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fqbuild.build()
    fq.lib()


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cstack(z):
    return np.stack([z.real, z.imag])


@pytest.fixture(scope="module")
def c3_full():
    w = W.config3()
    assert (w.S, w.n_frames, w.P, w.A, w.M, w.Ns) == (500_000, 100, 128 ** 3, 9, 1024, 1536)
    pl = Pipeline(w, **BENCH_STORAGE)
    pl.upload()
    pl.step()
    torch.cuda.synchronize()
    fq.fq_clutter_status(pl.ws_svd)
    yield w, pl
    del pl
    torch.cuda.empty_cache()


# (transmit, element) lines spread over the tilts, the array's corners, edges and centre
LINES = [(0, 0), (0, 1023), (1, 31), (2, 528), (3, 992), (4, 0), (4, 527), (4, 1023),
         (5, 300), (6, 777), (7, 33), (8, 511), (8, 1000)]


def test_c3_full_rf_sampled(c3_full):
    """RF of 13 (transmit, element) lines of frames 0 and 63 against the
    oracle on the same scatterers: the benchmark's BF16 records at the BF16
    bar, and the same frames synthesised in FP32 from the GPU's own
    advected positions at the FP32 bar."""
    w, pl = c3_full
    st, mt = W.segment_table(w), W.motion_table(w.motion)
    _, amp_eff = oracle.classify(w.p0, w.seg, st, len(w.segments), w.amp)
    assert np.array_equal(pl.pops[0].amp_eff.cpu().numpy(), amp_eff)
    idx = np.array([a * w.M + m for a, m in LINES])
    for f in (0, 63):
        pos = oracle.advect(w.p0, w.seg, w.flow, st, mt, f / w.prf)
        want = oracle.simulate_rf_lines(w.probe, w.tilt_x, w.tilt_y, idx, pos, amp_eff)
        got16 = pl.rf[f].float().reshape(w.A * w.M, w.Ns)[torch.from_numpy(idx).cuda()].cpu().numpy()
        assert rel_l2(got16, want) <= BF16_TOL
        rf32 = fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, pl.pops[0].pos[f:f + 1], pl.pops[0].amp_eff, 1)
        got = rf32[0].reshape(w.A * w.M, w.Ns)[torch.from_numpy(idx).cuda()].cpu().numpy()
        assert rel_l2(got, want) <= RF_TOL


@pytest.fixture(scope="module")
def c3_two_frames(c3_full):
    """FP32 RF of frames 0 and 1 of the full workload (GPU positions) and the
    oracle's rf2iq + DAS of the middle y-slice of the 128^3 grid on it."""
    w, pl = c3_full
    rf = fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, pl.pops[0].pos[0:2].contiguous(), pl.pops[0].amp_eff, 2)
    rf_h = rf.cpu().numpy()
    g = w.grid
    iy = 64
    sl = W.Grid(g.nx, 1, g.nz, g.x0, g.y0 + iy * g.dy, g.z0, g.dx, 0.0, g.dz, g.fnumber)
    want = oracle.beamform(w.probe, w.tilt_x, w.tilt_y, rf_h, sl)
    return w, rf, want, iy


def _slice(w, iq, iy):
    g = w.grid
    got = iq.float().cpu().numpy().reshape(g.ny, g.nz * g.nx, 2, 2)[iy]
    return got[..., 0] + 1j * got[..., 1]


def test_c3_full_das_sampled(c3_two_frames):
    """rf2iq + DAS over the full 128^3 grid (1024 elements, 9 tilts) on two
    frames: the middle y-slice (16384 voxels) against the oracle, with FP32
    channel IQ at the FP32 bar and with BF16 channel IQ (the benchmark's
    storage) at the BF16 bar."""
    w, rf, want, iy = c3_two_frames
    iq = fq.fq_beamform_das(w.probe, w.tilt_x, w.tilt_y, rf, 2, w.grid)
    assert rel_l2(cstack(_slice(w, iq, iy)), cstack(want)) <= RF_TOL
    del iq
    iq = fq.fq_beamform_das(w.probe, w.tilt_x, w.tilt_y, rf, 2, w.grid, ch_dtype=torch.bfloat16)
    assert rel_l2(cstack(_slice(w, iq, iy)), cstack(want)) <= BF16_TOL


def test_c3_full_das_f16_channels(c3_two_frames):
    """The same slice with FP16 RF and channel IQ (FP32 arithmetic): the FP16
    storage rounding (2^-11 relative) keeps the image within 1e-3."""
    w, rf, want, iy = c3_two_frames
    iq = fq.fq_beamform_das(w.probe, w.tilt_x, w.tilt_y, rf.half(), 2, w.grid, ch_dtype=torch.float16)
    assert rel_l2(cstack(_slice(w, iq, iy)), cstack(want)) <= 1e-3


def test_c3_full_clutter_properties(c3_full):
    """Properties of the full-size SVD filter with the energy cutoff: the
    eigenvalues sum to ||S||_F^2 and descend, k is the smallest count whose
    eigenvalues hold 90% of the energy, PD >= 0 and
    sum_p PD_p = (1/F) sum_{j >= k} lambda_j."""
    w, pl = c3_full
    iq = pl.iq.double()
    tot = float((iq ** 2).sum())
    lam = pl.eigvals.cpu().numpy()
    k = int(pl.k_used.item())
    pd = pl.pd.double().cpu().numpy()
    assert abs(lam.sum() - tot) <= 1e-4 * tot
    assert np.all(np.diff(lam) <= 1e-6 * lam[0])
    cum = np.cumsum(lam)
    k_want = int(np.argmax(cum >= w.energy_thresh * cum[-1])) + 1
    assert 1 <= k <= w.n_frames
    if abs(cum[k_want - 1] - w.energy_thresh * cum[-1]) > 1e-5 * cum[-1]:  # no near-tie at the threshold
        assert k == k_want
    assert pd.min() >= 0
    want = lam[k:].sum() / w.n_frames
    assert abs(pd.sum() - want) <= 1e-3 * want + 1e-6 * lam[0] / w.n_frames


@pytest.fixture(scope="module")
def c3_reduced():
    """A seeded subset of the 3D workload (20k scatterers of the tree and
    tissue, 16 frames, 32^3 voxels) through the whole oracle path."""
    w = W.shrink(W.config3(seed=3, n_frames=16), max_scat=20_000, grid_div=4)
    ref = oracle.pipeline(w, W.segment_table(w), W.motion_table(w.motion))
    return w, ref


def _run(w, **kw):
    pl = Pipeline(w, **kw)
    pd = pl.step_e2e().numpy().copy()
    torch.cuda.synchronize()
    fq.fq_clutter_status(pl.ws_svd)
    iq = pl.iq.float().cpu().numpy()
    return pl, pd, iq[..., 0] + 1j * iq[..., 1]


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_c3_reduced_whole_path_pd(c3_reduced, storage):
    """Whole path on the 3D subset with FP32 or FP16 RF / channel IQ storage
    (FP32 Casorati, FP32 arithmetic): IQ and power Doppler within their bars
    of the FP64 oracle, and the same energy cutoff."""
    w, ref = c3_reduced
    dt = torch.float32 if storage == "f32" else torch.float16
    pl, pd, S = _run(w, rf_dtype=dt, ch_dtype=dt, iq_dtype=torch.float32)
    assert int(pl.k_used.item()) == ref["k"]
    assert rel_l2(cstack(S), cstack(ref["S"])) <= (RF_TOL if storage == "f32" else 1e-3)
    assert rel_l2(pd, ref["pd"]) <= PD_TOL


def test_c3_reduced_whole_path_bf16_storage(c3_reduced):
    """The benchmark's storage (BF16 RF and channel IQ, FP32 Casorati) on the
    3D subset: RF and IQ within the BF16 bar of the FP64 oracle."""
    w, ref = c3_reduced
    pl, pd, S = _run(w, **BENCH_STORAGE)
    assert rel_l2(pl.rf.float().cpu().numpy(), ref["rf"]) <= BF16_TOL
    assert rel_l2(cstack(S), cstack(ref["S"])) <= BF16_TOL

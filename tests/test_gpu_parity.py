"""CUDA path vs the FP64 oracle, element by element, on the same seeded
inputs (through the C ABI).  Tolerances: integer / index work bit-exact;
RF and IQ relative L2 <= 1e-5 in FP32, <= 1e-2 with BF16 storage; power
Doppler relative L2 <= 1e-3; advected positions within 1 ulp of binary32."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq
from paper_2509_05464_gb300 import workload as W

pytestmark = pytest.mark.gpu

RF_TOL = 1e-5
BF16_TOL = 1e-2
PD_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fqbuild.build()
    fq.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.float().cpu().numpy() if t.dtype == torch.bfloat16 else t.cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def tables(w):
    return W.segment_table(w), W.motion_table(w.motion)


# --------------------------------------------------------------- a1 advect --
def _advect_cases():
    w2 = W.config2(n_scat=20_000, n_frames=3)
    w3 = W.config3(n_scat=20_000, n_frames=3)
    w1 = W.config1()
    w1.motion = W.Motion(vel=(3e-3, 3e-3, 3e-3), omega=(0.0, -0.2, 0.0), rot_center=(0.0, 0.0, 25e-3))
    return [(w2, 0.0, 1e-3), (w3, 0.0, 1e-3), (w1, 0.0, 1e-3), (w2, 7.3, 0.25)]


@pytest.mark.parametrize("case", range(4))
def test_advect_within_one_ulp(case):
    w, t0, dt = _advect_cases()[case]
    st, mt = tables(w)
    F = w.n_frames
    pos = host(fq.fq_advect_scatterers(dev(w.p0), dev(w.seg), dev(w.flow), w.segments, w.motion, t0, dt, F))
    for f in range(F):
        t = t0 + f * dt
        want = oracle.advect(w.p0, w.seg, w.flow, st, mt, t)
        ulp = np.spacing(np.abs(want).astype(np.float32))
        diff = np.abs(pos[f].astype(np.float64) - want.astype(np.float64))
        assert np.all(diff <= ulp), (f, float((diff / ulp).max()))
        assert np.mean(diff == 0) > 0.999


# --------------------------------------------------- a2 membership, binning --
def _near_wall_points(w, rng, n=4000):
    """points scattered within +-2% of the lumen walls of every segment"""
    pts = []
    for s in w.segments:
        k = n // max(1, len(w.segments))
        if s.kind == W.SEG_LINE:
            a = rng.uniform(-0.02, 1.02, k) * s.length
            r = s.radius * rng.uniform(0.98, 1.02, k)
            th = rng.uniform(0, 2 * math.pi, k)
            p = (np.array(s.p0)[:, None] + np.outer(s.a1, a) + np.outer(s.a2, r * np.cos(th))
                 + np.outer(s.a3, r * np.sin(th)))
        else:
            ph = rng.uniform(-0.05, s.phi1 + 0.05, k)
            r = s.radius * rng.uniform(0.98, 1.02, k)
            th = rng.uniform(0, 2 * math.pi, k)
            rr = s.arc_radius + r * np.cos(th)
            p = (np.array(s.p0)[:, None] + np.outer(s.a1, rr * np.cos(ph)) + np.outer(s.a2, rr * np.sin(ph))
                 + np.outer(s.a3, r * np.sin(th)))
        pts.append(p)
    return np.concatenate(pts, axis=1).astype(np.float32)


@pytest.mark.parametrize("cfg", ["c2", "c3"])
def test_classify_bit_exact(cfg):
    w = W.config2(n_scat=30_000, n_frames=1) if cfg == "c2" else W.config3(n_scat=30_000, n_frames=1)
    st, _ = tables(w)
    rng = np.random.default_rng(4)
    extra = _near_wall_points(w, rng)
    pos = np.concatenate([w.p0, extra], axis=1)
    seg = np.concatenate([w.seg, np.full(extra.shape[1], -1, np.int32)])
    amp = np.concatenate([w.amp, rng.standard_normal(extra.shape[1]).astype(np.float32)])
    # blood rows of p0 are zero; give them real positions (their t = 0 flow position)
    pos[:, :w.S] = oracle.advect(w.p0, w.seg, w.flow, st, W.motion_table(W.Motion()), 0.0)
    v_gpu, a_gpu = fq.fq_classify_scatterers(dev(pos), dev(seg), w.segments, dev(amp))
    v_ref, a_ref = oracle.classify(pos, seg, st, len(w.segments), amp)
    assert np.array_equal(host(v_gpu), v_ref)
    assert np.array_equal(host(a_gpu), a_ref)
    assert (v_ref[w.S:] >= 0).sum() > 100 and (v_ref[w.S:] < 0).sum() > 100


@pytest.mark.parametrize("S,B", [(0, 5), (1, 1), (4095, 7), (4096, 230), (4097, 230), (100_003, 230), (50_000, 8192)])
def test_bin_bit_exact(S, B):
    rng = np.random.default_rng(S + B)
    z0, dz = 0.5e-3, 0.1e-3
    z = rng.uniform(-1e-3, z0 + dz * B * 1.1, S).astype(np.float32)
    if S > 100:
        z[:40] = z[40:80]
        z[80] = np.float32(z0)
        z[81] = np.float32(z0 + 3 * dz)
    off_g, perm_g = fq.fq_bin_scatterers(dev(z) if S else torch.empty(0, device="cuda"), z0, dz, B)
    off_r, perm_r = oracle.bin_scatterers(z, z0, dz, B)
    assert np.array_equal(host(off_g), off_r)
    assert np.array_equal(host(perm_g)[:S], perm_r)


# ------------------------------------------------------------ a3 RF synthesis --
def _positions(w, frames):
    st, mt = tables(w)
    return np.stack([oracle.advect(w.p0, w.seg, w.flow, st, mt, f / w.prf) for f in frames])


def _rf_cases():
    c1 = W.config1()
    c2 = W.shrink(W.config2(n_scat=100_000, n_frames=2), max_scat=4000)
    c3 = W.shrink(W.config3(n_scat=50_000, n_frames=1), max_scat=500)
    return {"c1": (c1, [0, 5]), "c2": (c2, [0, 1]), "c3": (c3, [0])}


@pytest.mark.parametrize("cfg", ["c1", "c2", "c3"])
def test_rf_parity_fp32(cfg):
    w, frames = _rf_cases()[cfg]
    pos = _positions(w, frames).astype(np.float32)
    rf = host(fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, dev(pos), dev(w.amp), len(frames)))
    for i in range(len(frames)):
        want = oracle.simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos[i], w.amp)
        err = rel_l2(rf[i], want)
        assert err <= RF_TOL, (cfg, i, err)


@pytest.mark.parametrize("cfg", ["c1", "c2", "c3"])
@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_rf_parity_16bit(cfg, dt):
    """16-bit RF storage: binary32 delays and taps rounded on the FMA pipe
    (errors ~1e-4, below the storage rounding); FP16 (2^-11) within 1e-3,
    BF16 (2^-9) within the 1e-2 storage bar."""
    w, frames = _rf_cases()[cfg]
    pos = _positions(w, frames).astype(np.float32)
    t = torch.float16 if dt == "f16" else torch.bfloat16
    rf = host(fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, dev(pos), dev(w.amp), len(frames), out_dtype=t).float())
    for i in range(len(frames)):
        want = oracle.simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos[i], w.amp)
        err = rel_l2(rf[i], want)
        assert err <= (1e-3 if dt == "f16" else BF16_TOL), (cfg, dt, i, err)


def test_rf_static_tissue_base_and_bf16():
    """Alg. 1: RF_total = RF_tissue(frame 0) + RF_blood(frame f) through the
    rf_base input; BF16 storage within 1e-2."""
    w = W.config1()
    nt = w.n_tissue
    pos = _positions(w, [0, 3]).astype(np.float32)
    pos_t = np.ascontiguousarray(pos[:1, :, :nt])
    pos_b = np.ascontiguousarray(pos[:, :, nt:])
    base = fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, dev(pos_t), dev(w.amp[:nt]), 1)
    rf = host(fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, dev(pos_b), dev(w.amp[nt:]), 2, rf_base=base[0]))
    for i in range(2):
        want = oracle.simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos_t[0], w.amp[:nt])
        want = oracle.simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos_b[i], w.amp[nt:], rf=want, accumulate=True)
        assert rel_l2(rf[i], want) <= RF_TOL
    rf16 = host(fq.fq_simulate_rf(w.probe, w.tilt_x, w.tilt_y, dev(pos), dev(w.amp), 2, out_dtype=torch.bfloat16))
    want = oracle.simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos[1], w.amp)
    assert rel_l2(rf16[1], want) <= BF16_TOL


@pytest.mark.parametrize("route", ["quad", "pair", "wide_element", "three_cycle"])
def test_rf_kernel_routes(route):
    """Every RF kernel route against the oracle: the quad kernel (rows of
    whole quads), the paired kernel (rows of 6), and the general kernel for
    elements wider than the fitted directivity covers (k0 w / 2 > 5) and for
    a three-cycle pulse."""
    nx, pitch, width, nc = {"quad": (8, 0.3e-3, 0.3e-3, 2), "pair": (6, 0.3e-3, 0.3e-3, 2),
                            "wide_element": (8, 0.6e-3, 0.55e-3, 2), "three_cycle": (8, 0.3e-3, 0.3e-3, 3)}[route]
    fs = 20e6 if nc == 2 else 30e6
    p = W.Probe(nx, 1, pitch, pitch, width, width, 5e6, fs, 1540.0, 0.5, nc, 700)
    rng = np.random.default_rng(7)
    S = 600
    pos = np.stack([rng.uniform(-4e-3, 4e-3, S), np.zeros(S), rng.uniform(2e-3, 24e-3, S)]).astype(np.float32)
    amp = rng.standard_normal(S).astype(np.float32)
    tx = [-0.05, 0.0, 0.08]
    rf = host(fq.fq_simulate_rf(p, tx, [0.0] * 3, dev(pos[None]), dev(amp), 1))
    want = oracle.simulate_rf(p, tx, [0.0] * 3, pos, amp)
    assert rel_l2(rf[0], want) <= RF_TOL, route


@pytest.mark.parametrize("A,ns", [(1, 1024), (2, 2048), (5, 2048)])
def test_rf_quad_cta_shapes(A, ns):
    """The 4-element kernel at each of its CTA shapes: records of 16 KB (four
    256-thread CTAs per SM), 64 KB (two of 512) and 160 KB (one of 1024)."""
    p = W.Probe(8, 1, 0.1e-3, 0.1e-3, 0.1e-3, 0.1e-3, 15.6e6, 62.5e6, 1540.0, 0.5, 2, ns)
    rng = np.random.default_rng(A + ns)
    S = 300
    pos = np.stack([rng.uniform(-3e-3, 3e-3, S), np.zeros(S), rng.uniform(1e-3, 20e-3, S)]).astype(np.float32)
    amp = rng.standard_normal(S).astype(np.float32)
    tx = list(np.radians(np.linspace(-6.0, 6.0, A))) if A > 1 else [0.0]
    rf = host(fq.fq_simulate_rf(p, tx, [0.0] * A, dev(pos[None]), dev(amp), 1))
    want = oracle.simulate_rf(p, tx, [0.0] * A, pos, amp)
    assert rel_l2(rf[0], want) <= RF_TOL


def test_rf_quantum_extremes():
    """The 4-element kernel picks each record's integer quantum from an upper
    bound of the sum of |taps| per sample, so the int32 records cannot wrap:
    a coherent pile of 3000 scatterers at one point (the bound is the whole
    sum), one bright near-field scatterer among weak ones (its record's
    quantum follows the bright echo; the weak echoes elsewhere keep 1e-4 of
    their own norm), a large static base, and a single scatterer."""
    p = W.Probe(8, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 700)
    tx, ty = [-0.05, 0.0, 0.08], [0.0] * 3
    rng = np.random.default_rng(23)

    def run(pos, amp, base=None):
        got = fq.fq_simulate_rf(p, tx, ty, dev(pos[None]), dev(amp), 1,
                                rf_base=None if base is None else dev(base))
        want = oracle.simulate_rf(p, tx, ty, pos, amp, rf=None if base is None else base.astype(np.float64),
                                  accumulate=base is not None)
        return host(got)[0], want

    pile = np.tile(np.array([[1e-3], [0.0], [6e-3]], np.float32), (1, 3000))
    got, want = run(pile, np.ones(3000, np.float32))
    assert np.abs(want).max() > 1000.0 * np.abs(oracle.simulate_rf(p, tx, ty, pile[:, :1], np.ones(1, np.float32))).max() / 1.001
    assert rel_l2(got, want) <= RF_TOL

    S = 2000
    pos = np.stack([rng.uniform(-4e-3, 4e-3, S), np.zeros(S), rng.uniform(8e-3, 16e-3, S)]).astype(np.float32)
    pos[:, 0] = (0.0, 0.0, 0.4e-3)  # bright echo near t = 0.5 us
    amp = rng.standard_normal(S).astype(np.float32)
    amp[0] = 1000.0
    got, want = run(pos, amp)
    assert rel_l2(got, want) <= RF_TOL
    late = np.zeros(want.shape, bool)
    late[..., 150:] = True  # past the bright echo
    assert rel_l2(got[late], want[late]) <= 1e-4

    base = (1e4 * rng.standard_normal((3, 8, 700))).astype(np.float32)
    got, want = run(pos[:, 1:].copy(), amp[1:].copy(), base)
    assert rel_l2(got, want) <= RF_TOL
    assert rel_l2(got - base, want - base) <= 1e-3

    got, want = run(pos[:, 5:6].copy(), np.array([0.7], np.float32))
    assert rel_l2(got, want) <= RF_TOL


def test_rf_scatterer_groups_with_base():
    """FP32 records of more than 65536 scatterers are accumulated in groups
    with their own quanta and summed in FP32 (150k scatterers: three
    groups), with a static base added once: against the oracle, and the
    dense medium's error stays at the FP32 bar."""
    p = W.Probe(8, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 700)
    tx, ty = [-0.05, 0.0, 0.08], [0.0] * 3
    rng = np.random.default_rng(31)
    S = 150_000
    pos = np.stack([rng.uniform(-4e-3, 4e-3, S), rng.uniform(-1e-3, 1e-3, S),
                    rng.uniform(2e-3, 16e-3, S)]).astype(np.float32)
    amp = rng.standard_normal(S).astype(np.float32)
    base = (30.0 * rng.standard_normal((3, 8, 700))).astype(np.float32)
    got = host(fq.fq_simulate_rf(p, tx, ty, dev(pos[None]), dev(amp), 1, rf_base=dev(base)))[0]
    want = oracle.simulate_rf(p, tx, ty, pos, amp, rf=base.astype(np.float64), accumulate=True)
    assert rel_l2(got, want) <= RF_TOL
    got = host(fq.fq_simulate_rf(p, tx, ty, dev(pos[None]), dev(amp), 1))[0]
    want = oracle.simulate_rf(p, tx, ty, pos, amp)
    assert rel_l2(got, want) <= RF_TOL


def test_rf_edge_cases():
    """no scatterers -> zeros; scatterers whose echo straddles the record
    ends keep only the in-record samples."""
    p = W.Probe(8, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 300)
    z = torch.zeros((1, 3, 0), device="cuda")
    rf = host(fq.fq_simulate_rf(p, [0.0], [0.0], z, torch.zeros(0, device="cuda"), 1))
    assert not rf.any()
    # depth 0.05 mm (echo at t ~ 0) and ~11.5 mm (echo around the last sample)
    pos = np.array([[[0.1e-3, 0.0, -0.2e-3], [0.0, 0.0, 0.0], [0.05e-3, 11.53e-3, 11.6e-3]]], np.float32)
    amp = np.array([1.0, -2.0, 0.5], np.float32)
    rf = host(fq.fq_simulate_rf(p, [0.0], [0.0], dev(pos), dev(amp), 1))
    want = oracle.simulate_rf(p, [0.0], [0.0], pos[0], amp)
    assert np.abs(want[0, :, -3:]).max() > 0
    assert rel_l2(rf[0], want) <= RF_TOL


# --------------------------------------------------------- a4 rf2iq, a5 DAS --
def test_rf2iq_parity():
    p = W.Probe(4, 1, 0.1e-3, 0.1e-3, 0.1e-3, 0.1e-3, 15.6e6, 62.5e6, 1540.0, 0.5, 2, 1000)
    rng = np.random.default_rng(0)
    F, L = 3, 6
    rf = rng.standard_normal((F, L, p.n_samples)).astype(np.float32)
    iq = host(fq.fq_rf2iq(p, L, F, dev(rf)))  # [L][Ns][Fp][2]
    want = oracle.rf2iq(p, rf)  # [F][L][Ns] complex
    got = iq[:, :, :F, 0] + 1j * iq[:, :, :F, 1]  # [L][Ns][F]
    want = want.transpose(1, 2, 0)
    assert rel_l2(np.stack([got.real, got.imag]), np.stack([want.real, want.imag])) <= RF_TOL
    assert not iq[:, :, F:].any()


def _das_cases():
    c1 = W.config1(n_frames=3)
    c2 = W.shrink(W.config2(n_scat=100_000, n_frames=3), max_scat=3000, grid_div=4)
    c3 = W.shrink(W.config3(n_scat=50_000, n_frames=2), max_scat=300, grid_div=8)
    return {"c1": c1, "c2": c2, "c3": c3}


def _oracle_rf(w, frames):
    pos = _positions(w, frames).astype(np.float32)
    return np.stack([oracle.simulate_rf(w.probe, w.tilt_x, w.tilt_y, pos[i], w.amp) for i in range(len(frames))]
                    ).astype(np.float32)


@pytest.mark.parametrize("cfg", ["c1", "c2", "c3"])
def test_beamform_parity_fp32(cfg):
    w = _das_cases()[cfg]
    F = w.n_frames
    rf = _oracle_rf(w, range(F))
    iq = host(fq.fq_beamform_das(w.probe, w.tilt_x, w.tilt_y, dev(rf), F, w.grid))
    want = oracle.beamform(w.probe, w.tilt_x, w.tilt_y, rf, w.grid)
    got = iq[..., 0] + 1j * iq[..., 1]
    err = rel_l2(np.stack([got.real, got.imag]), np.stack([want.real, want.imag]))
    assert err <= RF_TOL, (cfg, err)


def test_beamform_bf16_storage():
    w = _das_cases()["c2"]
    F = w.n_frames
    rf = _oracle_rf(w, range(F))
    want = oracle.beamform(w.probe, w.tilt_x, w.tilt_y, rf, w.grid)
    iq = host(fq.fq_beamform_das(w.probe, w.tilt_x, w.tilt_y, dev(rf).bfloat16(), F, w.grid,
                                 ch_dtype=torch.bfloat16, iq_dtype=torch.bfloat16))
    got = iq[..., 0] + 1j * iq[..., 1]
    assert rel_l2(np.stack([got.real, got.imag]), np.stack([want.real, want.imag])) <= BF16_TOL


# --------------------------------------------------- a6-a8 clutter filter --
def _clutter(P, F, k, seed, gap=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((F, F)) + 1j * rng.standard_normal((F, F)))
    Uc, _ = np.linalg.qr(rng.standard_normal((P, k)) + 1j * rng.standard_normal((P, k)))
    L = (Uc * (gap * np.linspace(2.0, 1.0, k))) @ Q[:, :k].conj().T
    B = (rng.standard_normal((P, F)) + 1j * rng.standard_normal((P, F))) * 0.3
    return L + B


def cdev(S):
    return dev(np.stack([S.real, S.imag], axis=-1).astype(np.float32))


def cplx(t):
    a = host(t).astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("P,F", [(3000, 10), (3001, 64), (2048, 200), (100, 2)])
def test_gram_parity(P, F):
    rng = np.random.default_rng(P * F)
    S = (rng.standard_normal((P, F)) + 1j * rng.standard_normal((P, F))).astype(np.complex64).astype(np.complex128)
    G = cplx(fq.fq_casorati_gram(cdev(S)))
    want = oracle.gram(S)
    assert np.abs(G - want).max() <= 1e-5 * np.abs(want).max()


def _round_bf16(x):
    """binary32 -> bfloat16, round to nearest even (as float64)."""
    return torch.from_numpy(np.asarray(x, np.float32)).bfloat16().double().numpy()


def _round_tf32(x):
    """binary32 -> TF32 (10 explicit mantissa bits), round to nearest with
    ties away from zero, as the operand conversion cvt.rna.tf32.f32 does."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x1000) & 0xFFFFE000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _round_c(S, mode):
    r = _round_bf16 if mode == fq.FQ_GRAM_BF16 else _round_tf32
    return r(S.real) + 1j * r(S.imag)


def test_operand_rounding_helpers():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -11), 1.0 + 2.0 ** -11 + 2.0 ** -20])
    assert list(_round_bf16(x)) == [1.0, 1.0, 1.0 + 2.0 ** -6, -(1.0 + 2.0 ** -11) + 2.0 ** -11, 1.0]
    assert list(_round_tf32(x)) == [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -10),
                                    1.0 + 2.0 ** -10]


@pytest.mark.parametrize("mode", [2, 1], ids=["bf16", "tf32"])
@pytest.mark.parametrize("P,F", [(3000, 10), (3001, 64), (2048, 200), (100, 2), (5000, 300), (64, 512),
                                 (40000, 33)])
def test_gram_tensor_core_parity(mode, P, F):
    """tcgen05 Gram: the exact Gram of the operand-rounded input (products of
    BF16 / TF32 operands are exact in FP32), up to FP32 accumulation."""
    rng = np.random.default_rng(P * F + mode)
    S = (rng.standard_normal((P, F)) + 1j * rng.standard_normal((P, F))).astype(np.complex64).astype(np.complex128)
    ws = fq.workspace(fq.fq_gram_workspace_size(P, F, mode), torch.device("cuda"))
    G = cplx(fq.fq_casorati_gram(cdev(S), gram_mode=mode, ws=ws))
    fq.fq_clutter_status(ws)  # no timed-out wait
    want = oracle.gram(_round_c(S, mode))
    assert np.abs(G - want).max() <= 1e-5 * np.abs(want).max()
    off = G - np.diag(np.diag(G))
    assert np.array_equal(off, off.conj().T)  # lower triangle is the conjugate of the upper


def test_gram_tensor_core_bf16_input():
    rng = np.random.default_rng(77)
    S = rng.standard_normal((5000, 96)) + 1j * rng.standard_normal((5000, 96))
    Sb = cdev(S).bfloat16()
    Sq = cplx(Sb)
    for mode in (fq.FQ_GRAM_BF16, fq.FQ_GRAM_TF32):
        G = cplx(fq.fq_casorati_gram(Sb, gram_mode=mode))
        want = oracle.gram(Sq)
        assert np.abs(G - want).max() <= 1e-5 * np.abs(want).max()


@pytest.mark.parametrize("mode", [2, 1], ids=["bf16", "tf32"])
def test_clutter_svd_tensor_core_gram(mode):
    """The whole filter with the tensor-core Gram on FP32 input.  Rounding
    the Gram operand moves the clutter subspace; the tolerance adds to
    PD_TOL four times the PD change that this rounding alone causes in exact
    arithmetic (eigh of the FP64 Gram of the rounded input, FP64 projection
    of the unrounded one)."""
    k = 3
    S = _clutter(4096, 32, k, seed=11).astype(np.complex64).astype(np.complex128)
    r = fq.fq_clutter_svd(cdev(S), k_cut=k, gram_mode=mode)
    fq.fq_clutter_status(r["ws"])
    _, pd, sg, _ = oracle.svd_filter(S, k_cut=k)
    _, Vq = np.linalg.eigh(oracle.gram(_round_c(S, mode)))
    Vk = Vq[:, ::-1][:, :k]
    pd_q = np.mean(np.abs(S - (S @ Vk) @ Vk.conj().T) ** 2, axis=1)
    tol = PD_TOL + 4 * rel_l2(pd_q, pd)
    assert rel_l2(host(r["pd"]), pd) <= tol
    sq = np.linalg.svd(_round_c(S, mode), compute_uv=False)
    assert np.abs(host(r["eigvals"]) - sq ** 2).max() <= 2e-6 * sq[0] ** 2


# (1500, 80): a packed matrix under 48 KB that with the solver's static
# shared arrays still needs the opt-in (first in the list: a larger F would
# already have raised the attribute in this process)
@pytest.mark.parametrize("P,F,k", [(1500, 80, 2), (2000, 48, 3), (3000, 200, 2), (64, 8, 1), (50, 3, 1)])
def test_eig_against_oracle_svd(P, F, k):
    S = _clutter(P, F, k, seed=F).astype(np.complex64).astype(np.complex128)
    G64 = oracle.gram(S)
    lam, V, ws = fq.fq_hermitian_eig(cdev(G64))
    fq.fq_clutter_status(ws)
    lam, V = host(lam), cplx(V)
    _, Vo, sg = oracle.svd(S)
    lmax = sg[0] ** 2
    # FP32 Householder + QL: backward error ~ F eps ||G|| (eps = 2^-24)
    tol = max(2e-6, 2 * F * 2.0 ** -24)
    assert np.abs(lam - sg ** 2).max() <= tol * lmax
    assert np.all(np.diff(lam) <= 0)
    assert np.abs(V.conj().T @ V - np.eye(F)).max() <= max(1e-5, tol)
    assert np.abs(G64 @ V - V * lam).max() <= tol * lmax
    Pk = V[:, :k] @ V[:, :k].conj().T
    Po = Vo[:, :k] @ Vo[:, :k].conj().T
    assert np.abs(Pk - Po).max() <= 1e-5


def test_eig_degenerate_inputs():
    """rank-deficient (P < F) and a zero matrix: eigenvalues still match and
    the eigenvectors stay orthonormal."""
    rng = np.random.default_rng(3)
    S = (rng.standard_normal((5, 24)) + 1j * rng.standard_normal((5, 24))).astype(np.complex64).astype(np.complex128)
    G = oracle.gram(S)
    lam, V, ws = fq.fq_hermitian_eig(cdev(G))
    fq.fq_clutter_status(ws)
    lam, V = host(lam), cplx(V)
    want = np.sort(np.concatenate([np.linalg.svd(S, compute_uv=False) ** 2, np.zeros(19)]))[::-1]
    assert np.abs(lam - want).max() <= 2e-6 * want[0]
    assert np.abs(V.conj().T @ V - np.eye(24)).max() <= 1e-5
    lam, V, ws = fq.fq_hermitian_eig(cdev(np.zeros((6, 6), complex)))
    fq.fq_clutter_status(ws)
    assert not host(lam).any()
    assert np.abs(cplx(V).conj().T @ cplx(V) - np.eye(6)).max() <= 1e-6


@pytest.mark.parametrize("k_cut", [3, 0, -1, 32])
def test_clutter_svd_parity(k_cut):
    S = _clutter(4096, 32, 3, seed=11).astype(np.complex64).astype(np.complex128)
    r = fq.fq_clutter_svd(cdev(S), k_cut=k_cut, energy_thresh=0.9)
    fq.fq_clutter_status(r["ws"])
    S_f, pd, sg, k = oracle.svd_filter(S, k_cut=k_cut, energy_thresh=0.9)
    assert int(host(r["k"])[0]) == k
    assert np.abs(host(r["eigvals"]) - sg ** 2).max() <= 2e-6 * sg[0] ** 2
    if k == 32:
        assert not host(r["pd"]).any() and not host(r["iq_f"]).any()
        return
    assert rel_l2(host(r["pd"]), pd) <= PD_TOL
    got = cplx(r["iq_f"])
    assert rel_l2(np.stack([got.real, got.imag]), np.stack([S_f.real, S_f.imag])) <= PD_TOL


def test_clutter_svd_bf16_input():
    """BF16 Casorati input: both sides filter the same BF16-rounded matrix,
    so only the FP32 arithmetic of Gram, eigen-solver and projection
    separates them, and power Doppler meets its own bar."""
    S = _clutter(2048, 32, 2, seed=5).astype(np.complex64).astype(np.complex128)
    Sb = cdev(S).bfloat16()
    Sq = cplx(Sb)  # the BF16-rounded input both sides see
    r = fq.fq_clutter_svd(Sb, k_cut=2)
    _, pd, _, _ = oracle.svd_filter(Sq, k_cut=2)
    assert rel_l2(host(r["pd"]), pd) <= PD_TOL


def test_power_doppler_parity():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((5000, 37)) + 1j * rng.standard_normal((5000, 37))
    S = S.astype(np.complex64).astype(np.complex128)
    pd = host(fq.fq_power_doppler(cdev(S)))
    assert rel_l2(pd, oracle.power_doppler(S)) <= 1e-6

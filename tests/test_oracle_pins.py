"""Pins of the FP64 oracle against things other than itself: closed forms,
invariants, special cases that reduce to a library routine, and brute force
on tiny inputs.  CPU only.

Each test names the paper passage whose physics it relies on.
"""
import math

import numpy as np
import pytest
import scipy.signal
from scipy.spatial.transform import Rotation

import oracle
from paper_2509_05464_gb300 import workload as W


def probe(nx=16, ny=1, pitch=0.3e-3, f0=5e6, fs=80e6, ns=2048, width=None, alpha=0.5, ncyc=2):
    w = pitch if width is None else width
    return W.Probe(nx, ny, pitch, pitch, w, w, f0, fs, 1540.0, alpha, ncyc, ns)


def alpha_np(p):
    return p.alpha_db_cm_mhz * 100.0 / (20.0 / math.log(10.0))


def elem_x(p):
    return (np.arange(p.nx) - 0.5 * (p.nx - 1)) * p.pitch_x


# ---------------------------------------------------------------------------
# RF synthesis (Eq. 1 restated in time; Sec. 2.3, App. D)
# ---------------------------------------------------------------------------

def test_rf_single_scatterer_time_of_flight():
    """The echo envelope of one scatterer peaks at the geometric two-way time
    of flight (plane-wave transmit + spherical receive path, App. D)."""
    p = probe(nx=8, fs=160e6, ns=4096)
    xs, zs = 0.7e-3, 12.3e-3
    pos = np.array([[xs], [0.0], [zs]], np.float32)
    for theta in (0.0, math.radians(7.0), math.radians(-11.0)):
        rf = oracle.simulate_rf(p, np.array([theta]), np.zeros(1), pos, np.ones(1, np.float32))
        ex = elem_x(p)
        origin = np.min(ex * math.sin(theta))
        x, z = float(pos[0, 0]), float(pos[2, 0])
        for m in range(p.nx):
            tof = (x * math.sin(theta) + z * math.cos(theta) - origin + math.hypot(x - ex[m], z)) / p.c
            env = np.abs(scipy.signal.hilbert(rf[0, m]))
            k = int(np.argmax(env))
            y0, y1, y2 = env[k - 1], env[k], env[k + 1]
            frac = 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
            t_peak = (k + frac) / p.fs
            assert abs(t_peak - tof) * p.fs < 0.05, (m, t_peak * p.fs, tof * p.fs)


def test_rf_echo_energy_closed_form():
    """Sum_k RF[k]^2 for one scatterer right below an element equals
    A^2 fs * integral p(t)^2 dt, with integral = 3 T / 16 for a Hann-windowed
    tone, and A = R exp(-alpha f0 2z) / z (attenuation over the two-way path,
    1/r receive spreading, broadside directivity 1)."""
    p = probe(nx=4, fs=16 * 5e6, ns=4096)
    ex = elem_x(p)
    for m, z, R in ((1, 8e-3, 1.0), (1, 19e-3, -2.5), (2, 30e-3, 0.7)):
        pos = np.array([[ex[m]], [0.0], [z]], np.float32)
        x32, z32 = float(pos[0, 0]), float(pos[2, 0])
        assert x32 == np.float32(ex[m])
        rf = oracle.simulate_rf(p, np.zeros(1), np.zeros(1), pos, np.array([R], np.float32))
        r = math.hypot(x32 - ex[m], z32)
        path = z32 + r
        A = R * math.exp(-alpha_np(p) * p.f0 * 1e-6 * path) / r
        T = p.n_cycles / p.f0
        want = A * A * p.fs * 3.0 * T / 16.0
        got = float(np.sum(rf[0, m] ** 2))
        assert got == pytest.approx(want, rel=1e-6)


def test_rf_attenuation_ratio():
    """Two equal scatterers below one element at depths z1 < z2: peak ratio
    (z1/z2) exp(-alpha f0 (path2 - path1))."""
    p = probe(nx=2, fs=16 * 5e6, ns=8192)
    ex = elem_x(p)
    z1, z2 = 6e-3, 21e-3
    e = []
    for z in (z1, z2):
        pos = np.array([[ex[0]], [0.0], [z]], np.float32)
        rf = oracle.simulate_rf(p, np.zeros(1), np.zeros(1), pos, np.ones(1, np.float32))
        e.append(math.sqrt(np.sum(rf[0, 0] ** 2)))
    z1f, z2f = float(np.float32(z1)), float(np.float32(z2))
    want = (z1f / z2f) * math.exp(-alpha_np(p) * 5.0 * (2 * z2f - 2 * z1f))
    assert e[1] / e[0] == pytest.approx(want, rel=1e-8)


def test_rf_carrier_frequency():
    """The echo spectrum peaks near the centre frequency f0."""
    p = probe(nx=1, f0=7.8e6, fs=125e6, ns=8192)
    pos = np.array([[0.0], [0.0], [15e-3]], np.float32)
    rf = oracle.simulate_rf(p, np.zeros(1), np.zeros(1), pos, np.ones(1, np.float32))[0, 0]
    spec = np.abs(np.fft.rfft(rf, 1 << 16))
    f = np.fft.rfftfreq(1 << 16, 1 / p.fs)
    assert abs(f[np.argmax(spec)] - p.f0) < 0.15 * p.f0


def test_rf_directivity():
    """Element directivity D = sinc(k b sin(theta)) (App. D): broadside D = 1
    regardless of width; off axis the echo energy ratio between a wide and
    a point-like element is D^2."""
    z = 10e-3
    narrow = probe(nx=3, pitch=0.3e-3, width=1e-9, fs=80e6, ns=4096)
    wide = probe(nx=3, pitch=0.3e-3, width=0.3e-3, fs=80e6, ns=4096)
    for xs in (0.0, 2e-3, 6e-3):
        pos = np.array([[xs], [0.0], [z]], np.float32)
        e = []
        for pr in (narrow, wide):
            rf = oracle.simulate_rf(pr, np.zeros(1), np.zeros(1), pos, np.ones(1, np.float32))
            e.append(np.sum(rf[0, 1] ** 2))
        x, zz = float(pos[0, 0]), float(pos[2, 0])
        sin_t = x / math.hypot(x, zz)
        k = 2 * math.pi * wide.f0 / wide.c
        u = k * 0.5 * wide.width_x * sin_t
        D = 1.0 if u == 0 else math.sin(u) / u
        assert e[1] / e[0] == pytest.approx(D * D, rel=1e-9)
        if xs == 0.0:
            assert e[1] == pytest.approx(e[0], rel=1e-12)


def test_rf_superposition_and_static_tissue_reuse():
    """Weak scattering -> linear superposition (Sec. 2.2.1, App. D): the RF
    of a union of scatterer sets is the sum of their RFs, RF is linear in the
    reflection coefficients, and the static-tissue reuse of Alg. 1
    (RF_total = RF_tissue + RF_flow) is exact."""
    w = W.shrink(W.config1(), max_scat=300)
    p = w.probe
    rng = np.random.default_rng(5)
    pos = w.p0.copy()
    pos[0] += rng.uniform(-1e-4, 1e-4, pos.shape[1]).astype(np.float32)
    amp = w.amp
    half = pos.shape[1] // 2
    rf_all = oracle.simulate_rf(p, w.tilt_x, w.tilt_y, pos, amp)
    rf_a = oracle.simulate_rf(p, w.tilt_x, w.tilt_y, pos[:, :half].copy(), amp[:half].copy())
    rf_ab = oracle.simulate_rf(p, w.tilt_x, w.tilt_y, pos[:, half:].copy(), amp[half:].copy(),
                               rf=rf_a.copy(), accumulate=True)
    rf_b = oracle.simulate_rf(p, w.tilt_x, w.tilt_y, pos[:, half:].copy(), amp[half:].copy())
    scale = np.abs(rf_all).max()
    assert np.abs(rf_all - (rf_a + rf_b)).max() <= 1e-12 * scale
    assert np.abs(rf_all - rf_ab).max() <= 1e-12 * scale
    rf2 = oracle.simulate_rf(p, w.tilt_x, w.tilt_y, pos, (2 * amp).astype(np.float32))
    assert np.array_equal(rf2, 2 * rf_all)


def test_rf_mirror_symmetry():
    """x -> -x together with tilt -> -tilt mirrors the channels m -> M-1-m."""
    p = probe(nx=9, f0=5e6, fs=20e6, ns=1024)
    rng = np.random.default_rng(11)
    S = 40
    pos = np.stack([rng.uniform(-3e-3, 3e-3, S), np.zeros(S), rng.uniform(3e-3, 25e-3, S)]).astype(np.float32)
    amp = rng.standard_normal(S).astype(np.float32)
    th = np.radians([4.0, -9.0])
    rf = oracle.simulate_rf(p, th, np.zeros(2), pos, amp)
    mp = pos.copy()
    mp[0] = -mp[0]
    rfm = oracle.simulate_rf(p, -th, np.zeros(2), mp, amp)
    assert np.abs(rf - rfm[:, ::-1, :]).max() <= 1e-12 * np.abs(rf).max()


def test_rf_brute_force_all_samples():
    """Tiny case: evaluate the defining sum over *every* sample (no support
    truncation) in pure Python; matches the oracle's windowed loop."""
    p = probe(nx=2, ny=2, pitch=0.3e-3, f0=5e6, fs=20e6, ns=400)
    pos = np.array([[0.4e-3, -1.1e-3, 0.0], [0.2e-3, 0.9e-3, -0.3e-3], [5e-3, 8.7e-3, 12.1e-3]], np.float32)
    amp = np.array([1.0, -0.5, 2.0], np.float32)
    tx, ty = np.radians([3.0]), np.radians([-2.0])
    rf = oracle.simulate_rf(p, tx, ty, pos, amp)
    T = p.n_cycles / p.f0
    k0 = 2 * math.pi * p.f0 / p.c
    u = (math.sin(tx[0]), math.sin(ty[0]))
    u3 = math.sqrt(1 - u[0] ** 2 - u[1] ** 2)
    els = [((ix - 0.5) * p.pitch_x, (iy - 0.5) * p.pitch_y) for iy in range(2) for ix in range(2)]
    origin = min(u[0] * a + u[1] * b for a, b in els)
    want = np.zeros((4, p.n_samples))
    for m, (ex, ey) in enumerate(els):
        for s in range(3):
            x, y, z = (float(pos[d, s]) for d in range(3))
            r = math.sqrt((x - ex) ** 2 + (y - ey) ** 2 + z * z)
            path = u[0] * x + u[1] * y + u3 * z - origin + r
            tau = path / p.c
            ux = k0 * 0.5 * p.width_x * (x - ex) / r
            uy = k0 * 0.5 * p.width_y * (y - ey) / r
            D = (math.sin(ux) / ux) * (math.sin(uy) / uy)
            A = float(amp[s]) * D * math.exp(-alpha_np(p) * p.f0 * 1e-6 * path) / r
            for k in range(p.n_samples):
                t = k / p.fs - tau
                if abs(t) < T / 2:
                    want[m, k] += A * 0.5 * (1 + math.cos(2 * math.pi * t / T)) * math.cos(2 * math.pi * p.f0 * t)
    assert np.abs(rf[0] - want).max() <= 1e-12 * np.abs(want).max()


# ---------------------------------------------------------------------------
# rf2iq (Alg. 3 step 2.3.2.1)
# ---------------------------------------------------------------------------

def test_rf2iq_taps_are_a_unit_gain_lowpass():
    for f0, fs in ((5e6, 20e6), (15.6e6, 62.5e6), (7.8e6, 31.25e6)):
        h = oracle.rf2iq_taps(f0, fs)
        J = (len(h) - 1) // 2
        assert J == 2 * round(fs / f0)
        assert np.allclose(h, h[::-1], rtol=0, atol=1e-16)
        assert h.sum() == pytest.approx(1.0, abs=1e-14)
        j = np.arange(-J, J + 1)
        H = lambda f: abs(np.sum(h * np.exp(-2j * np.pi * f / fs * j)))
        assert H(2 * f0) < 0.05          # the 2 f0 image is rejected
        assert H(0.25 * f0) > 0.9        # the baseband passes


def test_rf2iq_matches_library_convolution():
    """IQ = 2 (RF * e^{-i w n}) convolved with h: compare with np.convolve."""
    p = probe(f0=15.6e6, fs=62.5e6, ns=700)
    rng = np.random.default_rng(3)
    rf = rng.standard_normal((3, p.n_samples)).astype(np.float32)
    iq = oracle.rf2iq(p, rf)
    h = oracle.rf2iq_taps(p.f0, p.fs)
    J = (len(h) - 1) // 2
    n = np.arange(p.n_samples)
    for l in range(3):
        mixed = rf[l].astype(np.float64) * np.exp(-2j * np.pi * p.f0 * n / p.fs)
        want = 2.0 * np.convolve(mixed, h)[J:J + p.n_samples]
        assert np.abs(iq[l] - want).max() <= 1e-12 * np.abs(want).max()


def test_rf2iq_pure_tone_gives_its_complex_amplitude():
    """A tone a cos(2 pi f0 n/fs + phi) demodulates to a e^{i phi} away from
    the record ends (up to the 2 f0 image leakage |H(2 f0)|)."""
    p = probe(f0=5e6, fs=20e6, ns=512)
    n = np.arange(p.n_samples)
    h = oracle.rf2iq_taps(p.f0, p.fs)
    J = (len(h) - 1) // 2
    leak = abs(np.sum(h * np.exp(-2j * np.pi * 2 * p.f0 / p.fs * np.arange(-J, J + 1))))
    for a, phi in ((1.0, 0.0), (2.5, 1.1), (0.3, -2.0)):
        rf = (a * np.cos(2 * np.pi * p.f0 * n / p.fs + phi)).astype(np.float32)[None]
        iq = oracle.rf2iq(p, rf)[0, J:-J]
        assert np.abs(iq - a * np.exp(1j * phi)).max() <= a * leak + 1e-6 * a


# ---------------------------------------------------------------------------
# DAS (Sec. 2.4.1, Alg. 3)
# ---------------------------------------------------------------------------

def _psf_setup(theta_list):
    p = probe(nx=48, pitch=0.3e-3, f0=5e6, fs=40e6, ns=2048)
    xs, zs = 0.45e-3, 14.2e-3
    pos = np.array([[xs], [0.0], [zs]], np.float32)
    rf = np.stack([oracle.simulate_rf(p, np.array([t]), np.zeros(1), pos, np.ones(1, np.float32))[0]
                   for t in theta_list])[None].astype(np.float32)
    return p, float(pos[0, 0]), float(pos[2, 0]), rf


def test_das_psf_peak_at_scatterer():
    """DAS of one scatterer peaks at the scatterer (T2), single and
    compounded transmits."""
    th = np.radians([-5.0, 0.0, 5.0])
    p, xs, zs, rf = _psf_setup(th)
    d = 0.025e-3
    g = W.Grid(41, 1, 41, xs - 20 * d, 0.0, zs - 20 * d, d, 0.0, d, 1.0)
    S = oracle.beamform(p, th, np.zeros(3), rf[:, :, :, :], g)[:, 0]
    img = np.abs(S).reshape(g.nz, g.nx)
    iz, ix = np.unravel_index(np.argmax(img), img.shape)
    assert abs(ix - 20) <= 1 and abs(iz - 20) <= 1

    def sub(a, b, c):
        return 0.5 * (a - c) / (a - 2 * b + c)
    fx = ix + sub(img[iz, ix - 1], img[iz, ix], img[iz, ix + 1])
    fz = iz + sub(img[iz - 1, ix], img[iz, ix], img[iz + 1, ix])
    assert abs(fx - 20) < 0.5 and abs(fz - 20) < 0.5


def _das_rows_by_hand(p, th, g):
    """The paper's per-transmit DAS matrices (Alg. 3 steps 2.2.1-2.2.2)
    built in the test from the definition: for every pixel and every
    element in the receive aperture, the two linear-interpolation weights at
    u = tau fs times the phase rotation e^{+i 2 pi f0 tau}.  Returns one
    dict {(row, col): value} per transmit."""
    ex = elem_x(p)
    xs = g.x0 + np.arange(g.nx) * g.dx
    zs = g.z0 + np.arange(g.nz) * g.dz
    mats = []
    for t in th:
        ent = {}
        origin = np.min(ex * math.sin(t))
        for iz, z in enumerate(zs):
            for ix, x in enumerate(xs):
                pidx = iz * g.nx + ix
                half = np.float32(z) * np.float32(0.5 / g.fnumber)
                for m in range(p.nx):
                    if abs(np.float32(x) - np.float32(ex[m])) > half:
                        continue
                    tau = (x * math.sin(t) + z * math.cos(t) - origin + math.hypot(x - ex[m], z)) / p.c
                    u = tau * p.fs
                    i = math.floor(u)
                    ph = u - i
                    if i < 0 or i + 1 >= p.n_samples:
                        continue
                    rot = np.exp(2j * math.pi * p.f0 * tau)
                    ent[(pidx, m * p.n_samples + i)] = (1 - ph) * rot
                    ent[(pidx, m * p.n_samples + i + 1)] = ph * rot
        mats.append(ent)
    return mats


def test_das_equals_explicit_das_matrix():
    """The paper precomputes one sparse DAS matrix per transmit and applies
    it to the vectorised IQ of every frame (Sec. 2.4.1, Alg. 3 steps
    2.2.1-2.4).  Matrices built in the test from the definition, applied
    with a library sparse product and averaged over transmits, reproduce
    the oracle's direct DAS sum; and the oracle's own explicit matrices
    equal the hand-built ones entry by entry."""
    import scipy.sparse as sp
    th = np.radians([-4.0, 3.0])
    p = probe(nx=12, pitch=0.3e-3, f0=5e6, fs=20e6, ns=512)
    rng = np.random.default_rng(2)
    F = 3
    rf = rng.standard_normal((F, 2, p.nx, p.n_samples)).astype(np.float32)
    g = W.Grid(7, 1, 9, -1.5e-3, 0.0, 4e-3, 0.5e-3, 0.0, 0.7e-3, 1.0)
    iq_ch = oracle.rf2iq(p, rf)
    direct = oracle.das(p, th, np.zeros(2), iq_ch, g)
    P = g.nz * g.nx
    hand = _das_rows_by_hand(p, th, g)
    out = np.zeros((P, F), complex)
    for a, ent in enumerate(hand):
        rows = [k[0] for k in ent]
        cols = [k[1] for k in ent]
        Mtx = sp.csr_matrix((list(ent.values()), (rows, cols)), shape=(P, p.nx * p.n_samples))
        for f in range(F):
            out[:, f] += Mtx @ iq_ch[f, a].reshape(-1)
    out /= len(th)
    assert np.abs(out - direct).max() <= 1e-12 * np.abs(direct).max()
    # the oracle's stored matrices: same entries, same values, every row
    row_ptr, col, val = oracle.das_matrix(p, th, np.zeros(2), g)
    for a, ent in enumerate(hand):
        got = {}
        for pidx in range(P):
            r = a * P + pidx
            for k in range(row_ptr[r], row_ptr[r + 1]):
                got[(pidx, int(col[k]))] = val[k]
        assert got.keys() == ent.keys()
        assert max(abs(got[k] - ent[k]) for k in ent) <= 1e-12


def _pulse(t, f0, T):
    return np.where(np.abs(t) < 0.5 * T, 0.5 * (1 + np.cos(2 * np.pi * t / T)) * np.cos(2 * np.pi * f0 * t), 0.0)


def _lowpass_taps(f0, fs):
    """rf2iq's filter from its stated definition: Hann-windowed ideal
    low-pass with cutoff f0, J = 2 round(fs/f0), unit DC gain."""
    J = 2 * round(fs / f0)
    j = np.arange(-J, J + 1)
    h = 2 * f0 / fs * np.sinc(2 * f0 / fs * j) * 0.5 * (1 + np.cos(np.pi * j / (J + 1)))
    return h / h.sum()


@pytest.mark.parametrize("ny", [1, 3])
def test_das_psf_peak_value_closed_form(ny):
    """Peak value of the compounded image of one scatterer (T2).  At the
    scatterer the DAS delay equals the echo's time of flight, so each
    (transmit, element) term is the echo amplitude A_{a,m} times the
    demodulated pulse h^(s) = 2 sum_j h_j p(s - j/fs) e^{-i 2 pi f0 (s - j/fs)}
    linearly interpolated at s = 0 between the samples s = -phi/fs and
    (1 - phi)/fs; the image value is (1/A) sum_a sum_m w_m of those terms
    (Sec. 2.4.1, Alg. 3 steps 2.3-2.4, with the echo model of App. D).
    Pins the absolute scale of rf2iq + DAS: a dropped 1/A, factor 2 or tap
    normalisation moves the peak."""
    p = probe(nx=10, ny=ny, pitch=0.3e-3, f0=5e6, fs=20e6, ns=1024)
    th_x = np.radians([-4.0, 0.0, 6.0])
    th_y = np.radians([0.0, 2.0, -3.0]) if ny > 1 else np.zeros(3)
    pos = np.array([[0.35e-3], [0.2e-3 if ny > 1 else 0.0], [9.1e-3]], np.float32)
    xs, ys, zs = (float(v) for v in pos[:, 0])
    R = np.array([1.7], np.float32)
    rf = oracle.simulate_rf(p, th_x, th_y, pos, R)[None].astype(np.float32)
    g = W.Grid(1, 1, 1, xs, ys, zs, 1e-4, 1e-4, 1e-4, 1.0)
    got = oracle.beamform(p, th_x, th_y, rf, g)[0, 0]

    ex = (np.arange(p.nx) - 0.5 * (p.nx - 1)) * p.pitch_x
    ey = (np.arange(ny) - 0.5 * (ny - 1)) * p.pitch_y
    h = _lowpass_taps(p.f0, p.fs)
    J = (len(h) - 1) // 2
    jj = np.arange(-J, J + 1)
    T = p.n_cycles / p.f0
    k0 = 2 * math.pi * p.f0 / p.c

    def hhat(s):
        tt = s - jj / p.fs
        return 2 * np.sum(h * _pulse(tt, p.f0, T) * np.exp(-2j * math.pi * p.f0 * tt))

    half = np.float32(zs) * np.float32(0.5 / g.fnumber)
    want = 0.0
    for a in range(3):
        sx, sy = math.sin(th_x[a]), math.sin(th_y[a])
        u = np.array([sx, sy, math.sqrt(1 - sx * sx - sy * sy)])
        origin = min(u[0] * x + u[1] * y for x in ex for y in ey)
        for iy in range(ny):
            for ix in range(p.nx):
                if abs(np.float32(xs) - np.float32(ex[ix])) > half:
                    continue
                if ny > 1 and abs(np.float32(ys) - np.float32(ey[iy])) > half:
                    continue
                dx, dy = xs - ex[ix], ys - ey[iy]
                r = math.sqrt(dx * dx + dy * dy + zs * zs)
                path = u @ np.array([xs, ys, zs]) - origin + r
                D = np.sinc(k0 * 0.5 * p.width_x * dx / r / math.pi)
                if ny > 1:
                    D *= np.sinc(k0 * 0.5 * p.width_y * dy / r / math.pi)
                amp = float(R[0]) * D * math.exp(-alpha_np(p) * p.f0 * 1e-6 * path) / r
                uu = path / p.c * p.fs
                phi = uu - math.floor(uu)
                want += amp * ((1 - phi) * hhat(-phi / p.fs) + phi * hhat((1 - phi) / p.fs))
    want /= 3
    assert abs(want) > 0
    assert abs(got - want) <= 1e-6 * abs(want), (got, want)


def test_das_mirror_symmetry():
    """Mirroring the channels and the tilts mirrors the image in x."""
    p = probe(nx=10, pitch=0.25e-3, f0=5e6, fs=20e6, ns=600)
    rng = np.random.default_rng(9)
    rf = rng.standard_normal((2, 2, p.nx, p.n_samples)).astype(np.float32)
    th = np.radians([2.0, -7.0])
    d = 2.0 ** -13
    g = W.Grid(9, 1, 6, -4 * d, 0.0, 5e-3, d, 0.0, 0.3e-3, 1.3)
    a = oracle.beamform(p, th, np.zeros(2), rf, g).reshape(g.nz, g.nx, 2)
    b = oracle.beamform(p, -th, np.zeros(2), rf[:, :, ::-1, :].copy(), g).reshape(g.nz, g.nx, 2)
    assert np.abs(a - b[:, ::-1, :]).max() <= 1e-12 * np.abs(a).max()


# ---------------------------------------------------------------------------
# SVD clutter filter + power Doppler (Sec. 2.4.2)
# ---------------------------------------------------------------------------

def _clutter_plus_blood(P, F, k, seed, gap=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((F, F)) + 1j * rng.standard_normal((F, F)))
    Vc, Vb = Q[:, :k], Q[:, k:]
    Uc, _ = np.linalg.qr(rng.standard_normal((P, k)) + 1j * rng.standard_normal((P, k)))
    sc = gap * np.linspace(2.0, 1.0, k)
    L = (Uc * sc) @ Vc.conj().T
    Xb = rng.standard_normal((P, F - k)) + 1j * rng.standard_normal((P, F - k))
    Xb -= Uc @ (Uc.conj().T @ Xb)  # blood orthogonal to the clutter in space as well as in time
    B = Xb @ Vb.conj().T * 0.1
    return L, B


def test_svd_filter_removes_rank_k_clutter_exactly():
    """S = L_k + B, clutter and blood orthogonal in space and in time, with a
    spectral gap: removing the k largest singular components returns B (T5)."""
    for P, F, k in ((200, 12, 2), (64, 9, 3), (150, 10, 1)):
        L, B = _clutter_plus_blood(P, F, k, seed=P + F)
        S_f, pd, sg, kk = oracle.svd_filter(L + B, k_cut=k)
        assert kk == k
        assert np.abs(S_f - B).max() <= 1e-10 * np.abs(L).max()
        assert np.allclose(pd, np.mean(np.abs(B) ** 2, axis=1), rtol=1e-8, atol=0)


def test_svd_singular_values_match_lapack():
    rng = np.random.default_rng(4)
    for P, F in ((300, 16), (40, 7), (5, 5)):
        S = rng.standard_normal((P, F)) + 1j * rng.standard_normal((P, F))
        US, V, sg = oracle.svd(S)
        ref = np.linalg.svd(S, compute_uv=False)
        assert np.allclose(sg, ref, rtol=1e-12, atol=0)
        assert np.allclose(US @ V.conj().T, S, atol=1e-12 * np.abs(S).max())
        assert np.allclose(V.conj().T @ V, np.eye(F), atol=1e-13)


def test_power_doppler_closed_form_and_energy_cutoff():
    """PD(p) = (1/F) sum_{j>k} sigma_j^2 |u_pj|^2 (LAPACK SVD), and the
    energy rule picks the smallest k reaching the threshold."""
    rng = np.random.default_rng(8)
    P, F = 120, 14
    S = (rng.standard_normal((P, F)) + 1j * rng.standard_normal((P, F))) * np.geomspace(30, 1, F)
    U, s, Vh = np.linalg.svd(S, full_matrices=False)
    for k in (0, 1, 3, F):
        _, pd, _, kk = oracle.svd_filter(S, k_cut=k)
        want = np.sum((s[k:] ** 2) * np.abs(U[:, k:]) ** 2, axis=1) / F
        assert kk == k
        assert np.allclose(pd, want, rtol=1e-9, atol=1e-12 * np.mean(np.abs(S) ** 2))
    for thr in (0.5, 0.9, 0.99):
        _, _, _, kk = oracle.svd_filter(S, k_cut=-1, energy_thresh=thr)
        c = np.cumsum(s ** 2) / np.sum(s ** 2)
        assert kk == int(np.argmax(c >= thr)) + 1
    S_f, pd, _, _ = oracle.svd_filter(S, k_cut=2)
    assert np.allclose(oracle.power_doppler(S_f), pd, rtol=1e-12)
    with pytest.raises(ValueError):
        oracle.svd_filter(S, k_cut=F + 1)


def test_gram_brute_force():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((33, 6)) + 1j * rng.standard_normal((33, 6))
    G = oracle.gram(S)
    want = np.zeros((6, 6), complex)
    for i in range(6):
        for j in range(6):
            for p in range(33):
                want[i, j] += np.conj(S[p, i]) * S[p, j]
    assert np.allclose(G, want, rtol=0, atol=1e-12)
    assert np.allclose(G, S.conj().T @ S, atol=1e-12)


# ---------------------------------------------------------------------------
# advection (Sec. 2.2.2) and tissue motion (Sec. 3.2)
# ---------------------------------------------------------------------------

def _one_line_vessel(R=0.4e-3, vmax=20e-3, L=30e-3):
    d = W._unit((1.0, 0.2, 0.5))
    sg = W.line_segment((-10e-3, 1e-3, 5e-3), d, L, R, vmax)
    return sg


def test_poiseuille_mean_speed_disc_and_stripe():
    """Mean Poiseuille speed over a uniformly sampled disc is vmax/2; over a
    planar stripe (2D) it is 2 vmax/3 (T4)."""
    sg = _one_line_vessel()
    rng = np.random.default_rng(0)
    for planar, want in ((False, 0.5), (True, 2.0 / 3.0)):
        n = 200_000
        ids, q, x1, x2 = W._blood_flow_coords(rng, [sg], [n], planar=planar)
        q[:] = 1e-3
        w = W.Workload("t", probe(), np.zeros(1), np.zeros(1), W.Grid(1, 1, 1, 0, 0, 0, 1, 1, 1),
                       [sg], W.Motion(), 1, 1.0, *W._assemble(np.zeros((3, 0)), np.zeros(0), ids, q, x1, x2,
                                                               np.ones(n)))
        st, mt = W.segment_table(w), W.motion_table(w.motion)
        t = 0.05
        a = oracle.advect(w.p0, w.seg, w.flow, st, mt, 0.0).astype(np.float64)
        b = oracle.advect(w.p0, w.seg, w.flow, st, mt, t).astype(np.float64)
        speed = ((b - a).T @ np.array(sg.a1)) / t
        sem = speed.std() / math.sqrt(n)
        assert abs(speed.mean() - want * sg.vmax) < 4 * sem + 1e-6 * sg.vmax


def test_blood_stays_in_lumen():
    """Blood trajectories stay inside the vessel lumen at every frame
    (Sec. 2.2.2), checked with an independent numpy distance computation."""
    w = W.config2(n_scat=20_000, n_frames=5)
    st, mt0 = W.segment_table(w), W.motion_table(W.Motion())
    blood = w.seg >= 0
    for t in (0.0, 0.37, 2.9):
        pos = oracle.advect(w.p0, w.seg, w.flow, st, mt0, t).astype(np.float64)
        for i, sg in enumerate(w.segments):
            sel = (w.seg == i)
            wv = pos[:, sel].T - np.array(sg.p0)
            x1, x2, x3 = wv @ np.array(sg.a1), wv @ np.array(sg.a2), wv @ np.array(sg.a3)
            rho = np.sqrt((np.hypot(x1, x2) - sg.arc_radius) ** 2 + x3 ** 2)
            assert rho.max() < sg.radius * (1 + 1e-5)
            ang = np.arctan2(x2, x1)
            assert ang.min() > -1e-6 and ang.max() < sg.phi1 + 1e-6
    assert blood.sum() > 0


def test_motion_closed_forms():
    """Steady translation P0 + V t (Sec. 3.2, V = (3,3,3) mm/s), steady
    rotation about (0,0,2.5 cm) against scipy's rotation, sinusoidal terms at
    quarter period, elastic gain 1 at the elastic centre (T10)."""
    rng = np.random.default_rng(7)
    S = 500
    p0 = np.stack([rng.uniform(-5e-3, 5e-3, S), rng.uniform(-5e-3, 5e-3, S),
                   rng.uniform(5e-3, 40e-3, S)]).astype(np.float32)
    seg = np.full(S, -1, np.int32)
    flow = np.zeros((3, S), np.float32)
    st = np.zeros((1, 24))
    t = 0.123
    m = W.Motion(vel=(3e-3, 3e-3, 3e-3))
    out = oracle.advect(p0, seg, flow, st, W.motion_table(m), t)
    want = p0.astype(np.float64) + np.array(m.vel)[:, None] * t
    assert np.abs(out - want).max() <= 2 * np.spacing(np.float32(0.05))
    # rotation V = (0, -w, 0) x (r - c): angular velocity vector (0, -w, 0)
    om = 0.4
    m = W.Motion(omega=(0.0, -om, 0.0), rot_center=(0.0, 0.0, 25e-3))
    out = oracle.advect(p0, seg, flow, st, W.motion_table(m), t).astype(np.float64)
    rot = Rotation.from_rotvec(np.array([0.0, -om * t, 0.0]))
    want = rot.apply(p0.astype(np.float64).T - [0, 0, 25e-3]).T + np.array([[0.0], [0.0], [25e-3]])
    assert np.abs(out - want).max() <= 2 * np.spacing(np.float32(0.05))
    # sinusoid: at a quarter period the displacement is A along dir
    m = W.Motion(amp=[80e-6], freq=[2.0], phase=[0.0], dir=[(0.0, 0.6, 0.8)],
                 elastic_grad=(0.0, 0.0, 30.0), elastic_center=(0.0, 0.0, 20e-3))
    out = oracle.advect(p0, seg, flow, st, W.motion_table(m), 0.125).astype(np.float64)
    gain = 1.0 + 30.0 * (p0[2].astype(np.float64) - 20e-3)
    want = p0 + np.outer([0.0, 0.6, 0.8], 80e-6 * gain)
    assert np.abs(out - want).max() <= 2 * np.spacing(np.float32(0.05))
    out = oracle.advect(p0, seg, flow, st, W.motion_table(m), 0.25).astype(np.float64)
    assert np.abs(out - p0).max() <= 2 * np.spacing(np.float32(0.05))


# ---------------------------------------------------------------------------
# vessel membership and depth binning
# ---------------------------------------------------------------------------

def test_classify_constructed_points():
    """Points built inside / outside each lumen by construction."""
    line = _one_line_vessel(R=0.5e-3, L=10e-3)
    arc = W.arc_segment((2e-3, 0.0, 12e-3), (1.0, 0.0, 0.0), (0.0, 0.0, 1.0), 4e-3, math.radians(120), 0.3e-3, 1e-2)
    w_segs = [line, arc]
    st = W.segment_table(W.Workload("t", probe(), np.zeros(1), np.zeros(1), W.Grid(1, 1, 1, 0, 0, 0, 1, 1, 1),
                                    w_segs, W.Motion(), 1, 1.0, np.zeros((3, 1)), np.zeros(1), np.zeros((3, 1)),
                                    np.zeros(1)))
    pts, want = [], []
    a1, a2, a3 = (np.array(v) for v in (line.a1, line.a2, line.a3))
    for s, r, exp in ((5e-3, 0.2e-3, 0), (0.5e-3, 0.49e-3, 0), (5e-3, 0.6e-3, -1), (-0.2e-3, 0.0, -1),
                      (10.3e-3, 0.0, -1)):
        pts.append(np.array(line.p0) + s * a1 + r * (0.6 * a2 + 0.8 * a3))
        want.append(exp)
    b1, b2, b3 = (np.array(v) for v in (arc.a1, arc.a2, arc.a3))
    for phi, dr, dz, exp in ((0.3, 0.0, 0.0, 1), (2.0, 0.25e-3, 0.0, 1), (1.0, 0.0, 0.29e-3, 1),
                             (2.2, 0.0, 0.0, -1), (-0.1, 0.0, 0.0, -1), (1.0, 0.35e-3, 0.0, -1)):
        rr = arc.arc_radius + dr
        pts.append(np.array(arc.p0) + rr * (math.cos(phi) * b1 + math.sin(phi) * b2) + dz * b3)
        want.append(exp)
    pos = np.array(pts, np.float64).T.astype(np.float32)
    S = pos.shape[1]
    seg = np.full(S, -1, np.int32)
    seg[0] = 1  # a blood scatterer keeps its own segment wherever it is
    want[0] = 1
    amp = np.arange(1, S + 1, dtype=np.float32)
    vessel, amp_out = oracle.classify(pos, seg, st, 2, amp)
    assert list(vessel) == want
    exp_amp = np.where((seg < 0) & (np.array(want) >= 0), 0.0, amp)
    assert np.array_equal(amp_out, exp_amp.astype(np.float32))


def test_bin_matches_stable_argsort():
    rng = np.random.default_rng(12)
    z = rng.uniform(-1e-3, 25e-3, 5000).astype(np.float32)
    z[:50] = z[50:100]  # ties
    z0, dz, B = 0.5e-3, 0.1e-3, 200
    off, perm = oracle.bin_scatterers(z, z0, dz, B)
    key = np.clip(np.floor((z.astype(np.float64) - z0) / dz), 0, B - 1).astype(np.int64)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=B))]))
    off0, perm0 = oracle.bin_scatterers(np.zeros(0, np.float32), z0, dz, B)
    assert off0.sum() == 0 and perm0.size == 0

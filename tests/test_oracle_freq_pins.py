"""Pins of the frequency-domain RF oracle (Eq. 1 evaluated per frequency,
Alg. 2 step 2.6) against the pulse's numerically integrated spectrum, the
time-domain oracle in the narrowband limit, and superposition.  CPU only."""
import math

import numpy as np
import scipy.integrate as si

import oracle
from paper_2509_05464_gb300 import workload as W


def pulse_spectrum_quad(f, f0, T):
    """S(f) = integral of p(t) e^{-i 2 pi f t} dt (p is even: a cosine integral)"""
    g = lambda t: 0.5 * (1 + math.cos(2 * math.pi * t / T)) * math.cos(2 * math.pi * f0 * t) * math.cos(2 * math.pi * f * t)
    return si.quad(g, -T / 2, T / 2, limit=200)[0]


def test_single_echo_spectrum():
    """with ns = N the output holds one full period; its DFT at bin j is
    N df S(f_j) A_j e^{-i 2 pi f_j tau}, A_j = D_j exp(-alpha f_j c tau) / r"""
    p = W.Probe(4, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 512)
    N = 512
    pos = np.array([[0.5e-3], [0.0], [8e-3]], np.float32)
    tilt = 0.1
    out = oracle.simulate_rf_freq(p, [tilt], [0.0], pos, np.array([1.0], np.float32), n_fft=N)[0, 2]
    X = np.fft.fft(out)
    df = p.fs / N
    T = p.n_cycles / p.f0
    ex = (np.arange(4) - 1.5) * p.pitch_x
    x, z = float(pos[0, 0]), float(pos[2, 0])
    origin = min(ex * math.sin(tilt))
    r = math.hypot(x - ex[2], z)
    tau = (x * math.sin(tilt) + z * math.cos(tilt) - origin + r) / p.c
    alpha = p.alpha_db_cm_mhz * 100 / (20 / math.log(10))
    for j in (1, 17, 64, 128, 200, 255):
        fj = j * df
        k = 2 * math.pi * fj / p.c
        arg = k * 0.5 * p.width_x * (x - ex[2]) / r
        D = math.sin(arg) / arg
        A = D * math.exp(-alpha * fj * 1e-6 * p.c * tau) / r
        want = N * df * pulse_spectrum_quad(fj, p.f0, T) * A * np.exp(-2j * math.pi * fj * tau)
        assert abs(X[j] - want) <= 1e-11 * np.abs(X).max(), j
    assert abs(X[N // 2]) <= 1e-9 * np.abs(X).max()  # no Nyquist term


def test_narrowband_limit_equals_time_domain():
    """without attenuation, with point-like elements and fs = 16 f0 (the
    pulse's spectrum beyond fs/2 is negligible) both restatements of Eq. 1
    give the same RF"""
    p = W.Probe(4, 1, 0.3e-3, 0.3e-3, 1e-9, 1e-9, 5e6, 80e6, 1540.0, 0.0, 2, 2048)
    rng = np.random.default_rng(0)
    pos = np.stack([rng.uniform(-2e-3, 2e-3, 5), np.zeros(5), rng.uniform(4e-3, 12e-3, 5)]).astype(np.float32)
    amp = rng.normal(size=5).astype(np.float32)
    f = oracle.simulate_rf_freq(p, [0.0, 0.05], [0.0, 0.0], pos, amp)
    t = oracle.simulate_rf(p, [0.0, 0.05], [0.0, 0.0], pos, amp)
    assert np.abs(f - t).max() <= 1e-3 * np.abs(t).max()


def test_superposition():
    p = W.Probe(3, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 256)
    pos = np.array([[0.2e-3, -0.4e-3], [0.0, 0.0], [3e-3, 4e-3]], np.float32)
    amp = np.array([1.0, -0.5], np.float32)
    both = oracle.simulate_rf_freq(p, [0.0], [0.0], pos, amp)
    a = oracle.simulate_rf_freq(p, [0.0], [0.0], pos[:, :1].copy(), amp[:1])
    b = oracle.simulate_rf_freq(p, [0.0], [0.0], pos[:, 1:].copy(), amp[1:])
    assert np.allclose(both, a + b, rtol=0, atol=1e-12 * np.abs(both).max())


# ---------------------------------------------------------------------------
# Transmit sum over elements (Eq. 1) and sub-elements (Eq. 2)
# ---------------------------------------------------------------------------

def _green(f, p, x, y, z, qx, qy, bx, by, matrix):
    """one sub-element's Green's function, written out from Eq. 1's terms"""
    d = math.sqrt((x - qx) ** 2 + (y - qy) ** 2 + z * z)
    k = 2 * math.pi * f / p.c
    sinc = lambda u: 1.0 if u == 0 else math.sin(u) / u
    D = sinc(k * bx * (x - qx) / d) * (sinc(k * by * (y - qy) / d) if matrix else 1.0)
    alpha = p.alpha_db_cm_mhz * 100 / (20 / math.log(10))
    return D * math.exp(-alpha * f * 1e-6 * d) / d * np.exp(-1j * k * d)


def test_single_element_transmit_spectrum():
    """One transmitting element (weight 2.5) and one receiving element, one
    scatterer: the DFT of the record over one period is N df S(f_j) R
    W e^{-i 2 pi f_j dtau} g_tx(f_j) g_rx(f_j), with the steering delay of
    the transmitting element (Eq. 1: weight, delay, spherical propagation,
    attenuation and directivity on each leg)."""
    p = W.Probe(5, 1, 0.3e-3, 0.3e-3, 0.25e-3, 0.25e-3, 5e6, 20e6, 1540.0, 0.5, 2, 512)
    N = 512
    pos = np.array([[0.6e-3], [0.0], [7e-3]], np.float32)
    R = float(np.float32(0.8))  # the amplitude both sides see
    tilt = 0.12
    apod = np.zeros(5)
    apod[1] = 2.5
    out = oracle.simulate_rf_pfield(p, [tilt], [0.0], apod, pos, np.array([R], np.float32), n_sub=1, n_fft=N)[0, 3]
    X = np.fft.fft(out)
    df = p.fs / N
    T = p.n_cycles / p.f0
    ex = (np.arange(5) - 2.0) * p.pitch_x
    x, z = float(pos[0, 0]), float(pos[2, 0])
    dtau = (ex[1] * math.sin(tilt) - min(ex * math.sin(tilt))) / p.c
    for j in (1, 23, 64, 128, 200, 255):
        fj = j * df
        gt = _green(fj, p, x, 0.0, z, ex[1], 0.0, 0.5 * p.width_x, 0.5 * p.width_y, False)
        gr = _green(fj, p, x, 0.0, z, ex[3], 0.0, 0.5 * p.width_x, 0.5 * p.width_y, False)
        want = N * df * pulse_spectrum_quad(fj, p.f0, T) * R * 2.5 * np.exp(-2j * math.pi * fj * dtau) * gt * gr
        assert abs(X[j] - want) <= 1e-10 * np.abs(X).max(), j


def test_transmit_weights_superpose():
    """The record is linear in the transmit weights (Eq. 1 sums the
    elements' fields): weights a + b give the sum of the two records."""
    p = W.Probe(4, 2, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 20e6, 1540.0, 0.5, 2, 200)
    rng = np.random.default_rng(4)
    pos = np.stack([rng.uniform(-1e-3, 1e-3, 3), rng.uniform(-0.5e-3, 0.5e-3, 3),
                    rng.uniform(3e-3, 5e-3, 3)]).astype(np.float32)
    amp = rng.normal(size=3).astype(np.float32)
    wa, wb = rng.uniform(0, 1, 8), rng.uniform(-1, 1, 8)
    args = ([0.05, -0.02], [0.0, 0.03])
    ab = oracle.simulate_rf_pfield(p, *args, wa + wb, pos, amp, n_sub=2)
    a = oracle.simulate_rf_pfield(p, *args, wa, pos, amp, n_sub=2)
    b = oracle.simulate_rf_pfield(p, *args, wb, pos, amp, n_sub=2)
    assert np.abs(ab - a - b).max() <= 1e-12 * np.abs(ab).max()


def test_sub_elements_reach_the_far_field_limit():
    """v sub-elements of width w / v with the sub-element directivity sum to
    the whole element's directivity in the far field (the array factor of
    the sub-elements times their own sinc is sinc(k w/2 sin theta)); the
    near-field difference falls as 1/d: halving it when the scatterer's
    distance doubles.  One element transmits, one receives."""
    p = W.Probe(3, 1, 0.6e-3, 0.6e-3, 0.6e-3, 0.6e-3, 5e6, 20e6, 1540.0, 0.0, 2, 2048)
    apod = np.array([0.0, 1.0, 0.0])
    diffs = []
    for z in (8e-3, 16e-3, 32e-3):  # echoes well inside the 102 us record
        pos = np.array([[1.5e-3 * z / 10e-3], [0.0], [z]], np.float32)
        one = oracle.simulate_rf_pfield(p, [0.0], [0.0], apod, pos, np.ones(1, np.float32), n_sub=1)[0, 1]
        five = oracle.simulate_rf_pfield(p, [0.0], [0.0], apod, pos, np.ones(1, np.float32), n_sub=5)[0, 1]
        diffs.append(np.linalg.norm(five - one) / np.linalg.norm(one))
    assert diffs[0] < 0.06
    assert 0.45 < diffs[1] / diffs[0] < 0.55 and 0.45 < diffs[2] / diffs[1] < 0.55, diffs


def test_steered_full_aperture_arrival_time():
    """Every element transmitting with its steering delay builds the tilted
    wavefront: the echo of a scatterer on the array axis, deep compared with
    the aperture, peaks at the plane-wave time of flight
    (u . r - min u . e + |r - e_m|) / c (the envelope peak within 0.25
    sample; a single element's spherical wave would arrive ~1 sample later
    at this tilt and depth)."""
    import scipy.signal
    p = W.Probe(32, 1, 0.3e-3, 0.3e-3, 0.3e-3, 0.3e-3, 5e6, 40e6, 1540.0, 0.0, 2, 1024)
    pos = np.array([[0.0], [0.0], [15e-3]], np.float32)
    ex = (np.arange(32) - 15.5) * p.pitch_x
    for tilt in (0.0, math.radians(6.0)):
        rf = oracle.simulate_rf_pfield(p, [tilt], [0.0], np.ones(32), pos, np.ones(1, np.float32))[0]
        z = float(pos[2, 0])
        for m in (0, 16, 31):
            env = np.abs(scipy.signal.hilbert(rf[m]))
            k = int(np.argmax(env))
            y0, y1, y2 = env[k - 1], env[k], env[k + 1]
            t_peak = (k + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)) / p.fs
            tof = (z * math.cos(tilt) - min(ex * math.sin(tilt)) + math.hypot(ex[m], z)) / p.c
            assert abs(t_peak - tof) * p.fs < 0.25, (tilt, m, (t_peak - tof) * p.fs)

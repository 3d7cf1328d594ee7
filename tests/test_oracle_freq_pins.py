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

"""Pins of the post-processing / quality oracle (Sec. 5.2 display
compression, Sec. 6.1 MIPs, Sec. 5.3 MSE / PSNR / SSIM) against closed
forms and an independent library route.  CPU only."""
import numpy as np
import scipy.signal

from oracle import post


def test_compress_closed_forms():
    a = np.array([1.0, 0.1, 0.01, 1e-4, 0.0, -3.0])
    # amplitudes: 0, -20, -40, -80 dB over a 60 dB range; zero and negative -> 0
    assert np.allclose(post.compress(a, 20.0, 60.0), [1.0, 2 / 3, 1 / 3, 0.0, 0.0, 0.0], atol=1e-15)
    # powers: 10 log10
    p = np.array([4.0, 2.0, 0.4])
    want = (10 * np.log10(p / 4.0) + 60.0) / 60.0
    assert np.allclose(post.pd_display(p, 60.0), want, atol=1e-15)
    assert not post.compress(np.zeros(5), 20.0, 60.0).any()
    # scale invariance of the display
    x = np.random.default_rng(0).rayleigh(1.0, 100)
    assert np.allclose(post.compress(7.5 * x, 20.0, 75.0), post.compress(x, 20.0, 75.0), atol=1e-14)


def test_bmode_is_the_envelope_in_db():
    rng = np.random.default_rng(1)
    S = rng.normal(size=(50, 3)) + 1j * rng.normal(size=(50, 3))
    b = post.bmode(S, 2, 75.0)
    env = np.abs(S[:, 2])
    k = np.argmax(env)
    assert b[k] == 1.0
    j = np.argmin(env)
    assert np.isclose(b[j], max(0.0, (20 * np.log10(env[j] / env[k]) + 75.0) / 75.0))


def test_mip_of_a_point_volume():
    vol = np.full((5, 6, 7), 0.25)
    vol[3, 1, 4] = 9.0  # z, y, x
    mx = post.mip(vol, 0)   # along x -> [nz][ny]
    my = post.mip(vol, 1)   # along y -> [nz][nx]
    mz = post.mip(vol, 2)   # along z -> [ny][nx]
    assert mx.shape == (5, 6) and my.shape == (5, 7) and mz.shape == (6, 7)
    for m, idx in ((mx, (3, 1)), (my, (3, 4)), (mz, (1, 4))):
        assert m[idx] == 9.0
        assert np.count_nonzero(m == 9.0) == 1 and np.all(m[m != 9.0] == 0.25)


def test_mse_psnr_closed_forms():
    rng = np.random.default_rng(2)
    y = rng.uniform(0, 1, (20, 30))
    x = y + 0.05
    assert np.isclose(post.mse(x, y), 0.0025, rtol=1e-12)
    assert np.isclose(post.psnr(x, y), 10 * np.log10(1 / 0.0025), rtol=1e-12)
    assert np.isclose(post.psnr(2 * x, 2 * y, L=2.0), post.psnr(x, y), rtol=1e-12)


def test_ssim_identity_and_constant_images():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (24, 20))
    assert np.isclose(post.ssim(x, x), 1.0, atol=1e-12)
    a, b = 0.3, 0.7
    C1 = 0.01 ** 2
    got = post.ssim(np.full((15, 15), a), np.full((15, 15), b))
    assert np.isclose(got, (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)
    # window weights: Gaussian, sigma 1.5, normalised
    w = post.gaussian_window()
    assert w.shape == (11, 11) and np.isclose(w.sum(), 1.0)
    assert np.isclose(w[5, 6] / w[5, 5], np.exp(-1 / (2 * 1.5 ** 2)))


def test_ssim_matches_the_convolution_route():
    """the per-window loop equals the same statistics from valid-mode 2D
    convolutions (scipy.signal) of x, y, x^2, y^2, xy with the window"""
    rng = np.random.default_rng(4)
    y = rng.uniform(0, 1, (30, 26))
    x = np.clip(y + rng.normal(0, 0.1, y.shape), 0, 1)
    w = post.gaussian_window()[::-1, ::-1]  # convolution flips the kernel
    f = lambda im: scipy.signal.convolve2d(im, w, mode="valid")
    mx, my = f(x), f(y)
    sx, sy, sxy = f(x * x) - mx * mx, f(y * y) - my * my, f(x * y) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    m = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2))
    assert np.isclose(post.ssim(x, y), m.mean(), rtol=1e-12)
    assert post.ssim(x, y) < 1.0

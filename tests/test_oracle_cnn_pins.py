"""Pins of the learned-filter oracle (oracle/cnn.py) against facts that do
not come from it: the impulse response of a convolution is its kernel;
single-channel results equal scipy.ndimage.correlate with zero padding; the
backward pass is the adjoint of the forward pass and the network gradient
matches central finite differences.  CPU."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import cnn


def test_tap_table():
    assert cnn.N_TAPS == 45 and len(set(cnn.TAPS)) == 45
    for t, (dt, dz, dx) in enumerate(cnn.TAPS):
        assert t == (dt + 2) * 9 + (dz + 1) * 3 + (dx + 1)
    # 97,920 weights in the 2-32-32-32-2 network
    assert sum(45 * a * b for a, b in zip(cnn.CHANNELS[:-1], cnn.CHANNELS[1:])) == 97920


def test_impulse_response_is_the_kernel():
    rng = np.random.default_rng(0)
    w = rng.standard_normal((45, 2, 3))
    x = np.zeros((7, 5, 6, 2))
    f0, z0, x0, ci = 3, 2, 2, 1
    x[f0, z0, x0, ci] = 1.0
    y = cnn.conv3d(x, w, np.zeros(3))
    seen = np.zeros(y.shape[:3], bool)
    for t, (dt, dz, dx) in enumerate(cnn.TAPS):
        # y[v] = sum_t x[v + d_t] w_t: the impulse at u shows at v = u - d_t
        v = (f0 - dt, z0 - dz, x0 - dx)
        assert np.array_equal(y[v], w[t, ci])
        seen[v] = True
    assert not y[~seen].any()


def test_single_channel_equals_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((9, 6, 7, 1))
    w = rng.standard_normal((45, 1, 1))
    k = np.zeros((5, 3, 3))
    for t, (dt, dz, dx) in enumerate(cnn.TAPS):
        k[dt + 2, dz + 1, dx + 1] = w[t, 0, 0]
    want = ndimage.correlate(x[..., 0], k, mode="constant", cval=0.0)
    got = cnn.conv3d(x, w, np.zeros(1))[..., 0]
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_backward_is_the_adjoint():
    """<dy, conv(x, w)> is bilinear: its derivative along any direction of
    x, w or b is the inner product with the returned gradient, exactly."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 4, 4, 2))
    w = rng.standard_normal((45, 2, 3))
    b = rng.standard_normal(3)
    dy = rng.standard_normal((5, 4, 4, 3))
    gx, gw, gb = cnn.conv3d_backward(x, w, dy)
    L = lambda x_, w_, b_: float(np.sum(dy * cnn.conv3d(x_, w_, b_)))
    for _ in range(3):
        ex, ew, eb = rng.standard_normal(x.shape), rng.standard_normal(w.shape), rng.standard_normal(b.shape)
        assert L(x + ex, w, b) - L(x, w, b) == pytest.approx(np.sum(gx * ex), rel=1e-10)
        assert L(x, w + ew, b) - L(x, w, b) == pytest.approx(np.sum(gw * ew), rel=1e-10)
        assert L(x, w, b + eb) - L(x, w, b) == pytest.approx(np.sum(gb * eb), rel=1e-10)


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    chans = (2, 4, 4, 2)
    params = cnn.init_params(rng, chans)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    x = rng.standard_normal((6, 4, 5, 2))
    target = rng.standard_normal((6, 4, 5, 2))
    loss, grads = cnn.backward(cnn.forward(x, params), params, target)
    assert loss == pytest.approx(cnn.mse(cnn.forward(x, params)[-1], target))
    eps = 1e-6
    for l in range(len(params)):
        w, b = params[l]
        for which, arr in (("w", w), ("b", b)):
            d = rng.standard_normal(arr.shape)
            def loss_at(s):
                p = [(ww.copy(), bb.copy()) for ww, bb in params]
                if which == "w":
                    p[l] = (w + s * d, b)
                else:
                    p[l] = (w, b + s * d)
                return cnn.mse(cnn.forward(x, p)[-1], target)
            fd = (loss_at(eps) - loss_at(-eps)) / (2 * eps)
            g = grads[l][0] if which == "w" else grads[l][1]
            assert np.sum(g * d) == pytest.approx(fd, rel=1e-5, abs=1e-12)


def test_power_doppler_of_a_rotating_phasor():
    F = 16
    ph = np.linspace(0, 5, F)
    y = np.zeros((F, 2, 3, 2))
    y[..., 0] = (1.5 * np.cos(ph))[:, None, None]
    y[..., 1] = (1.5 * np.sin(ph))[:, None, None]
    assert np.allclose(cnn.power_doppler(y), 2.25)

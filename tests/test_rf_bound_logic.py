"""The tap bound that sets the 4-element RF kernel's integer quantum, checked
in FP64 on the CPU against the sums it must bound (no GPU).  For one element
pair and one plane-wave transmit: every scatterer adds |amp| D_b / r_s at the
sample nearest its binary32 delay of the pair's segment point plus half a
pitch (r_s = distance to the segment between the two elements, D_b the
directivity bound at the ends of the pair's argument range); the window sum
over 2 floor(half_w + pitch fs / 2c + 0.52) + 1 samples must be at least the
sum of |amp| |D| / r over the echoes whose support |t - u| < half_w covers the
sample, for both elements (the pulse is bounded by 1, the attenuation by 1 for
echoes after t = 0)."""
import math

import numpy as np


def sinc(u):
    return np.sinc(u / np.pi)


def d_bound(u):
    t = u * u
    return 1.0 - t / 6.0 + t * t / 120.0


def check_bound(x, z, amp, tilt, loose=None, width=0.1e-3):
    c, fs, f0, n_cycles, pitch = 1540.0, 62.5e6, 15.6e6, 2, 0.1e-3
    K = fs / c
    hw = n_cycles * fs / (2.0 * f0)
    kbx = math.pi * f0 / c * width
    win = int(math.floor(hw + 0.5 * pitch * K + 0.52))
    ns = 2048
    xe = np.array([0.35e-3, 0.45e-3])  # the pair's elements
    origin = min(-6.35e-3 * math.sin(tilt), 6.35e-3 * math.sin(tilt))
    ptx = x * math.sin(tilt) + z * math.cos(tilt) - origin

    # the bound, with the binary32 steps of the kernel
    xs = np.clip(x, xe[0], xe[1])
    rs = np.hypot(x - xs, z)
    d = np.maximum(d_bound(kbx * np.abs(x - xs) / rs), d_bound(kbx))
    b = amp * d / rs
    u_mid = ((ptx * K).astype(np.float32) + (rs * K).astype(np.float32) + np.float32(0.5 * pitch * K)).astype(np.float32)
    kp = np.rint(u_mid).astype(np.int64)
    bins = np.zeros(ns + 2 * win)
    ok = (kp + win >= 0) & (kp + win < ns + 2 * win)
    np.add.at(bins, kp[ok] + win, b[ok])
    # sample t: bins t .. t + 2 win, with the kernel's margin for rounding of the amplitudes
    bound = np.convolve(bins, np.ones(2 * win + 1), mode="valid") * (1.0 + 2.0 ** -7)
    assert bound.shape == (ns,)

    for e in range(2):
        r = np.hypot(x - xe[e], z)
        u = (ptx + r) * K
        a = amp * np.abs(sinc(kbx * (x - xe[e]) / r)) / r
        actual = np.zeros(ns)
        lo = np.floor(u - hw).astype(np.int64) + 1
        for j in range(int(2 * hw) + 2):
            t = lo + j
            inside = (np.abs(t - u) < hw) & (t >= 0) & (t < ns)
            np.add.at(actual, t[inside], a[inside])
        assert actual.max() > 0
        assert np.all(bound >= actual), (e, float((actual - bound).max()))
        if loose is not None:  # not grossly loose where the echoes are dense
            busy = actual > 0.5 * actual.max()
            assert np.median(bound[busy] / actual[busy]) < loose


def test_window_bound_covers_every_sample():
    rng = np.random.default_rng(17)
    S = 20000
    check_bound(rng.uniform(-7.5e-3, 7.5e-3, S), rng.uniform(0.05e-3, 21.5e-3, S), np.abs(rng.standard_normal(S)),
                math.radians(4.0), loose=4.0)


def test_window_bound_single_echoes():
    """one scatterer at a time, where no other echo's slack can hide a
    misplaced bound: broadside, steep lateral angles either side of the pair,
    and between the two elements near the surface"""
    for x, z, tilt in ((0.4e-3, 10e-3, 0.0), (7.5e-3, 0.3e-3, 0.1), (-7.5e-3, 0.2e-3, -0.1),
                       (0.4e-3, 0.06e-3, 0.05), (3e-3, 1e-3, -0.1), (-2e-3, 20e-3, 0.1)):
        check_bound(np.array([x]), np.array([z]), np.array([1.0]), tilt)
    # an element wide enough (k0 w / 2 = 4.5) that the directivity bound is not
    # monotone over the pair's range of arguments (4.27 and 3.18 here)
    check_bound(np.array([0.5e-3]), np.array([0.05e-3]), np.array([1.0]), 0.0, width=0.1415e-3)

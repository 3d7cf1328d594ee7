"""FP64 oracle of the learned clutter filter (test infrastructure only).

The network is four 3D convolution layers over an ensemble volume laid out
channels-last as ``[F][Z][X][C]`` (frames, depth, lateral, channels):
2 -> 32 -> 32 -> 32 -> 2 channels, kernels of 5 frames x 3 x 3 pixels,
zero "same" padding, a bias per output channel, ReLU after the first three
layers.  The input channels are the real and imaginary parts of the
normalised IQ, the output the estimated blood IQ; power Doppler is the
mean over frames of its squared magnitude.  Training minimises the mean
squared error against the blood-only IQ.  (The paper names the future-work
direction -- filters learned from simulated ensembles that resist motion --
in Sec. 1 and Sec. 4; the architecture is the one this library implements.)

Convention (cross-correlation, as deep-learning frameworks use it):

    y[v, o] = b[o] + sum_t sum_i x[v + d_t, i] w[t, i, o]

over the 45 tap offsets d_t = (dt, dz, dx), dt in -2..2, dz, dx in -1..1,
tap index t = (dt + 2) * 9 + (dz + 1) * 3 + (dx + 1); x is 0 outside the
volume.  Everything is numpy in float64 and written from these
definitions: one shifted copy of the input per tap and a matrix product.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dt, dz, dx) for dt in range(-2, 3) for dz in range(-1, 2) for dx in range(-1, 2)]
N_TAPS = len(TAPS)
CHANNELS = (2, 32, 32, 32, 2)


def shift(x: np.ndarray, d) -> np.ndarray:
    """s[f, z, x] = x[f + dt, z + dz, x + dx], 0 where that is outside."""
    dt, dz, dx = d
    F, Z, X = x.shape[:3]
    out = np.zeros_like(x)
    fs, fd = (slice(dt, F), slice(0, F - dt)) if dt >= 0 else (slice(0, F + dt), slice(-dt, F))
    zs, zd = (slice(dz, Z), slice(0, Z - dz)) if dz >= 0 else (slice(0, Z + dz), slice(-dz, Z))
    xs, xd = (slice(dx, X), slice(0, X - dx)) if dx >= 0 else (slice(0, X + dx), slice(-dx, X))
    out[fd, zd, xd] = x[fs, zs, xs]
    return out


def conv3d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [F, Z, X, Cin], w [45, Cin, Cout], b [Cout] -> [F, Z, X, Cout]."""
    y = np.zeros(x.shape[:3] + (w.shape[2],))
    for t, d in enumerate(TAPS):
        y += shift(x, d) @ w[t]
    return y + b


def conv3d_backward(x: np.ndarray, w: np.ndarray, dy: np.ndarray):
    """Gradients of sum(dy * conv3d(x, w, b)) with respect to x, w and b."""
    dx = np.zeros_like(x, dtype=np.float64)
    dw = np.zeros_like(w, dtype=np.float64)
    for t, d in enumerate(TAPS):
        xs = shift(x, d)
        dw[t] = xs.reshape(-1, x.shape[3]).T @ dy.reshape(-1, dy.shape[3])
        # y[v] gets x[v + d] w: x[u] feeds y[u - d]
        dx += shift(dy, tuple(-k for k in d)) @ w[t].T
    db = dy.reshape(-1, dy.shape[3]).sum(axis=0)
    return dx, dw, db


def init_params(rng: np.random.Generator, channels=CHANNELS):
    """He-normal weights (fan-in 45 Cin), zero biases."""
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        w = rng.standard_normal((N_TAPS, cin, cout)) * np.sqrt(2.0 / (N_TAPS * cin))
        params.append((w, np.zeros(cout)))
    return params


def forward(x: np.ndarray, params):
    """Activations of every layer: acts[0] = x, acts[l + 1] = layer l output
    (after ReLU for the first three)."""
    acts = [x]
    for l, (w, b) in enumerate(params):
        y = conv3d(acts[-1], w, b)
        if l < len(params) - 1:
            y = np.maximum(y, 0.0)
        acts.append(y)
    return acts


def mse(y: np.ndarray, target: np.ndarray) -> float:
    return float(np.mean((y - target) ** 2))


def backward(acts, params, target):
    """Loss and gradients [(dw, db) per layer] of mse(acts[-1], target)."""
    y = acts[-1]
    dy = 2.0 * (y - target) / y.size
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        dx, dw, db = conv3d_backward(acts[l], w, dy)
        grads[l] = (dw, db)
        if l > 0:
            dy = dx * (acts[l] > 0.0)  # ReLU of the previous layer
    return mse(y, target), grads


def power_doppler(y: np.ndarray) -> np.ndarray:
    """[F, Z, X, 2] (re, im) -> [Z, X] mean over frames of |y|^2."""
    return np.mean(y[..., 0] ** 2 + y[..., 1] ** 2, axis=0)

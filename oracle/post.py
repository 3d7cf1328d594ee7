"""FP64 oracle of the post-processing and quality module (test
infrastructure only): display compression, B-mode, maximum-intensity
projections and the image-quality metrics.

Sec. 5.2: B-mode and power-Doppler images are logarithmically compressed
and shown over a dynamic range (75 dB B-mode, 60 dB uPDI in Sec. 6.1);
Sec. 6.1 shows maximum-intensity projections of 3D uPDI volumes; Sec. 5.3
scores reconstructions against ground truth by MSE, PSNR and SSIM.  The
paper gives no formulas; this library reads them as:

    compress(a; g, DR) = clip((g log10(a / max a) + DR) / DR, 0, 1)
        g = 20 for amplitudes (B-mode envelope |S|), 10 for powers (PD);
        a <= 0 maps to 0, an all-zero image to all 0.
    bmode(S, f; DR) = compress(|S[:, f]|; 20, DR)
    mip(V, axis) = max of V along the axis (the other axes keep their order)
    MSE = mean (x - y)^2, PSNR = 10 log10(L^2 / MSE)
    SSIM = mean over the valid positions (no padding) of
           ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2))
        with the weighted statistics of an 11 x 11 Gaussian window
        (sigma 1.5, weights normalised to sum 1), C1 = (0.01 L)^2,
        C2 = (0.03 L)^2 (Wang, Bovik, Sheikh and Simoncelli, 2004).
"""
from __future__ import annotations

import numpy as np


def compress(a, g, dr_db):
    a = np.asarray(a, np.float64)
    m = a.max() if a.size else 0.0
    out = np.zeros_like(a)
    if m <= 0.0:
        return out
    pos = a > 0.0
    out[pos] = np.clip((g * np.log10(a[pos] / m) + dr_db) / dr_db, 0.0, 1.0)
    return out


def bmode(S, frame, dr_db=75.0):
    """S complex [P][F] -> [P] in [0, 1]"""
    return compress(np.abs(np.asarray(S)[:, frame]), 20.0, dr_db)


def pd_display(pd, dr_db=60.0):
    return compress(pd, 10.0, dr_db)


def mip(vol, axis):
    """vol [nz][ny][nx]; axis 0 = x, 1 = y, 2 = z (numpy axes 2, 1, 0)"""
    return np.asarray(vol, np.float64).max(axis={0: 2, 1: 1, 2: 0}[axis])


def gaussian_window(size=11, sigma=1.5):
    r = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-(r * r) / (2.0 * sigma * sigma))
    w = np.outer(g, g)
    return w / w.sum()


def mse(x, y):
    d = np.asarray(x, np.float64) - np.asarray(y, np.float64)
    return float(np.mean(d * d))


def psnr(x, y, L=1.0):
    return float(10.0 * np.log10(L * L / mse(x, y)))


def ssim(x, y, L=1.0, size=11, sigma=1.5):
    """mean SSIM over the valid window positions, from the definition: for
    every position the window's weighted means, variances and covariance
    (a plain loop over positions with a matrix product per window)"""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    w = gaussian_window(size, sigma)
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    H, W = x.shape
    vals = []
    for i in range(H - size + 1):
        for j in range(W - size + 1):
            a = x[i:i + size, j:j + size]
            b = y[i:i + size, j:j + size]
            mx, my = np.sum(w * a), np.sum(w * b)
            sx = np.sum(w * a * a) - mx * mx
            sy = np.sum(w * b * b) - my * my
            sxy = np.sum(w * a * b) - mx * my
            vals.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2)))
    return float(np.mean(vals))

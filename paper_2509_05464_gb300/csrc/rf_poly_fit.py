"""Writes rf_poly.cuh: the polynomial coefficients the RF kernels use for
the element directivity sin(u)/u and for sin x, cos x of the first pulse
tap.

Each polynomial is the Chebyshev interpolant of its function on the stated
interval (degree n, n + 1 Chebyshev points), a near-minimax fit, converted
to monomial form in v = t - t0 (t = u^2 or x^2) and rounded to binary32:

    sinc(u) = sin(u) / u   ~ S(u^2 - 12.5),  |u| <= 5      (degree 7)
    sin(x)                 ~ x P(x^2),       |x| <= 0.8    (degree 3)
    cos(x)                 ~ Q(x^2),         |x| <= 0.8    (degree 4)

Centring the sinc variable halves the rounding error of its binary32
Horner evaluation (the partial sums stay small).

Run ``python rf_poly_fit.py`` in this directory to regenerate the header;
``check()`` returns the FP64 approximation errors and the errors of the
binary32 Horner evaluation that the kernels perform.
"""
from __future__ import annotations

import os

import numpy as np
from numpy.polynomial import chebyshev as cheb
from numpy.polynomial import polynomial as poly

SINC_UMAX = 5.0
TAP_XMAX = 0.8
SPECS = {
    # name: (function of t, t range, degree, centre t0)
    "kSincPoly": (lambda t: _sinc_sqrt(t), SINC_UMAX ** 2, 7, SINC_UMAX ** 2 / 2),
    "kSinPoly": (lambda t: _sinc_sqrt(t), TAP_XMAX ** 2, 3, 0.0),
    "kCosPoly": (lambda t: np.cos(np.sqrt(t)), TAP_XMAX ** 2, 4, 0.0),
}
HEADER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rf_poly.cuh")


def _sinc_sqrt(t):
    """sin(sqrt t) / sqrt t, 1 at t = 0"""
    t = np.asarray(t, np.float64)
    r = np.sqrt(np.maximum(t, 1e-300))
    return np.where(t > 0, np.sin(r) / r, 1.0)


def fit(f, tmax: float, deg: int, t0: float) -> np.ndarray:
    """Monomial coefficients (lowest first, in v = t - t0) of the degree-deg
    Chebyshev interpolant of f on t in [0, tmax]."""
    dom = [-t0, tmax - t0]
    c = cheb.Chebyshev.interpolate(lambda v: f(v + t0), deg, domain=dom)
    return c.convert(kind=poly.Polynomial, domain=dom, window=dom).coef


def coefficients() -> dict:
    return {name: fit(f, tmax, deg, t0).astype(np.float32) for name, (f, tmax, deg, t0) in SPECS.items()}


def horner_f32(coef: np.ndarray, t: np.ndarray) -> np.ndarray:
    """binary32 Horner evaluation with fused multiply-adds (each step
    rounded once from its exact FP64 value, as a binary32 FMA does)"""
    t32 = np.asarray(t, np.float32)
    r = np.full(t32.shape, coef[-1], np.float32)
    for c in coef[-2::-1]:
        r = (r.astype(np.float64) * t32.astype(np.float64) + np.float64(c)).astype(np.float32)
    return r


def check(n: int = 20001) -> dict:
    """{name: (max |error| of the binary32 coefficients in FP64,
               max |error| of the binary32 Horner evaluation)}"""
    out = {}
    co = coefficients()
    for name, (f, tmax, _, t0) in SPECS.items():
        t = np.linspace(0.0, tmax, n)
        want = f(t)
        c64 = co[name].astype(np.float64)
        e64 = float(np.max(np.abs(np.polyval(c64[::-1], t - t0) - want)))
        v32 = (t.astype(np.float64) - np.float64(np.float32(t0))).astype(np.float32)  # one rounding, as an FMA
        e32 = float(np.max(np.abs(horner_f32(co[name], v32).astype(np.float64) - want)))
        out[name] = (e64, e32)
    return out


def render() -> str:
    lines = ["// Generated by rf_poly_fit.py: Chebyshev-interpolant coefficients",
             "// (lowest degree first, in v = t - t0 with t = u^2 or x^2), rounded to binary32.",
             "#pragma once", "", "namespace fqpoly {", "",
             f"constexpr float kSincUMax = {SINC_UMAX!r}f;",
             f"constexpr float kTapXMax = {TAP_XMAX!r}f;",
             f"constexpr float kSincCentre = {SPECS['kSincPoly'][3]!r}f;"]
    for name, c in coefficients().items():
        lines.append(f"// {name}0 .. {name}{len(c) - 1}")
        for i, v in enumerate(c):
            lines.append(f"constexpr float {name}{i} = {float(v):.9e}f;")
    lines += ["", "}  // namespace fqpoly", ""]
    return "\n".join(lines)


if __name__ == "__main__":
    with open(HEADER, "w") as fh:
        fh.write(render())
    for k, (e64, e32) in check().items():
        print(f"{k}: FP64 error {e64:.2e}, binary32 Horner error {e32:.2e}")

"""The fitted polynomials of the RF kernels (directivity sinc, first-tap
sin/cos): the committed header is what the fit writes, and the binary32
evaluation meets the error bounds the kernels rely on."""
import importlib.util
import os

import numpy as np

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2509_05464_gb300", "csrc")


def _fit():
    spec = importlib.util.spec_from_file_location("rf_poly_fit", os.path.join(CSRC, "rf_poly_fit.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_header_is_generated():
    m = _fit()
    with open(os.path.join(CSRC, "rf_poly.cuh")) as fh:
        assert fh.read() == m.render()


def test_error_bounds():
    err = _fit().check()
    assert err["kSincPoly"][1] <= 2e-7
    assert err["kSinPoly"][1] <= 6e-8
    assert err["kCosPoly"][1] <= 6e-8


def test_against_closed_forms():
    """spot values: sinc(pi) = 0, sinc(pi / 2) = 2 / pi, sin and cos at pi / 4"""
    m = _fit()
    c = m.coefficients()
    t0 = np.float32(m.SPECS["kSincPoly"][3])

    def sinc(u):
        return float(m.horner_f32(c["kSincPoly"], np.array([np.float32(u * u) - t0]))[0])

    assert abs(sinc(np.pi)) <= 2e-7
    assert abs(sinc(np.pi / 2) - 2 / np.pi) <= 2e-7
    assert abs(sinc(0.0) - 1.0) <= 2e-7
    x = np.pi / 4
    s = x * float(m.horner_f32(c["kSinPoly"], np.array([x * x]))[0])
    co = float(m.horner_f32(c["kCosPoly"], np.array([x * x]))[0])
    assert abs(s - np.sqrt(0.5)) <= 1e-7 and abs(co - np.sqrt(0.5)) <= 1e-7


def test_sinc_upper_bound():
    """the RF kernel bounds |sin(u)/u| on |u| <= 5 by 1 - u^2/6 + u^4/120 (the
    alternating series truncated after a positive term); the bound must hold
    on the whole range and be tight where the directivity is near 1"""
    u = np.linspace(0.0, 5.0, 500_001)
    t = u * u
    bound = 1.0 - t / 6.0 + t * t / 120.0
    s = np.abs(np.sinc(u / np.pi))
    assert (bound - s).min() >= -1e-15
    assert (bound / s)[u <= 2.0].max() < 1.03

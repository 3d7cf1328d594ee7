"""The C-ABI library builds, loads and exports every entry point that
include/fq.h declares; argument validation answers without touching the
GPU; the Python binding fails loudly when the library is missing.  CPU."""
import ctypes as C
import os
import re

import pytest

from paper_2509_05464_gb300 import build as fqbuild
from paper_2509_05464_gb300 import fq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fq_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libfq():
    fqbuild.build()
    return fq.lib()


def test_exports_every_declared_symbol(libfq):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(libfq, n)]
    assert not missing, missing


def test_info_calls(libfq):
    assert fq.version() >= 100
    assert libfq.fq_status_string(0) == b"FQ_OK"
    assert libfq.fq_status_string(7) == b"FQ_ERR_NUMERICAL"
    assert fq.frame_pad(1) == 16 and fq.frame_pad(200) == 208 and fq.frame_pad(16) == 16


def test_argument_validation_without_gpu(libfq):
    # null descriptors / bad sizes are rejected before any CUDA call
    assert libfq.fq_simulate_rf(None, None, None, None, 0, 1, None, 0, None, None) == 1
    assert b"null" in libfq.fq_last_error()
    p = fq.Probe(64, 1, 3e-4, 3e-4, 3e-4, 3e-4, 5e6, 20e6, 1540.0, 0.5, 2, 100000)
    tx_arr = (C.c_double * 1)(0.0)
    tx = fq.Tx(1, tx_arr, tx_arr)
    assert libfq.fq_simulate_rf(C.byref(p), C.byref(tx), None, None, 0, 1, None, 0, C.c_void_p(16), None) == 2
    p.n_samples = 1024
    # a dtype code outside fq_dtype
    assert libfq.fq_simulate_rf(C.byref(p), C.byref(tx), None, None, 0, 1, None, 7, C.c_void_p(16), None) == 8
    assert libfq.fq_simulate_rf(C.byref(p), C.byref(tx), None, None, 0, 1, None, 0, C.c_void_p(2), None) == 3
    n = C.c_size_t(0)
    assert libfq.fq_clutter_svd_workspace_size(65536, 200, 0, C.byref(n)) == 0 and n.value > 0
    # k_cut > F
    assert libfq.fq_clutter_svd(C.c_void_p(256), 0, 100, 8, 9, 0.9, 0, None, None, None, None,
                                C.c_void_p(256), n.value, None) == 1
    assert libfq.fq_bin_scatterers(None, 10, 0.0, 1e-4, 0, None, None, None, 0, None) == 2
    # unknown gram_mode; the tensor-core modes size their own scratch
    assert libfq.fq_casorati_gram(C.c_void_p(256), 0, 100, 8, 7, C.c_void_p(256), C.c_void_p(256), 1 << 20,
                                  None) == 1
    sizes = []
    for mode in (0, 1, 2):
        assert libfq.fq_gram_workspace_size(65536, 200, mode, C.byref(n)) == 0
        sizes.append(n.value)
    # BF16 operands take half the bytes of TF32 ones; 2F x P operand copy at least
    assert sizes[2] >= 400 * 65536 * 2 and sizes[1] >= 400 * 65536 * 4 and sizes[1] > sizes[2]
    assert libfq.fq_gram_workspace_size(65536, 200, 3, C.byref(n)) == 1
    assert libfq.fq_clutter_svd_workspace_size(65536, 200, 2, C.byref(n)) == 0 and n.value > sizes[2]


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(fq, "_lib", None)
    monkeypatch.setattr(fq, "LIB_PATH", "/nonexistent/libfq.so")
    with pytest.raises(fq.FqError):
        fq.lib()

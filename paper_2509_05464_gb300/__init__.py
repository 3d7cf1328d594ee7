"""GB300-native (sm_103a) uPDI hot path of 3D-FQFlow (arXiv 2509.05464).

The compute path lives in a C-ABI shared library (``include/fq.h``) built from
the CUDA sources in ``csrc/``.  ``paper_2509_05464_gb300.fq`` is the thin
Python binding (ctypes; torch tensors supply device memory and streams).
Importing this package does not load the library; the first call into
``fq`` does, and fails loudly if the library is missing.
"""
__all__ = ["fq", "workload"]

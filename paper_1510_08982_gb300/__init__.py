"""heat1d: GB300-native synchronous and asynchronous FTCS solver for the 1D
heat equation (Lee & Bhattacharya, arXiv:1510.08982).

The compute path is the CUDA library ``libheat1d.so`` (sm_103a) behind a C ABI
declared in ``include/heat1d.h``; ``paper_1510_08982_gb300.heat1d`` is the thin
ctypes binding with the same names.  Importing this package loads nothing;
the library is loaded on first use and a missing library is an error (there is
no CPU fallback).
"""
__all__ = ["heat1d", "inputs"]

"""CPU oracle for the 1D heat-equation FTCS update (arXiv:1510.08982).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library and its Python binding) never imports, links or runs anything here,
and this package never imports the product path.

The arithmetic lives in plain C (``heat1d_oracle.c``), built with gcc and
``-ffp-contract=off`` so that the only fused multiply-add is the one written out
(``fma(r, (uR - 2u) + uL, u)``, the order of the printed kernels in Section 4).
This module only compiles it, loads it with ctypes and marshals numpy arrays.

Functions (all return new numpy arrays; they raise ``OracleError`` on a
non-zero status from C):

* ``sync(u0, r, c1, cN, K, dtype)``      -- Section 2, Eq. (eqn:sync), Dirichlet ends.
* ``async_replay(u0, r, c1, cN, S, q, K, trace, dtype)`` -- Section 3, Eq. (eqn:async),
  the switched system driven by a given delay trace.
* ``adjoint(u0, r, c1, cN, K, u_obs, S, q, trace)`` -- FP64 gradient of
  0.5*||u(K) - u_obs||^2 with respect to u(0) and r.
* ``sync_periodic(u0, r, K, dtype)``, ``async_periodic(u0, r, S, q, K, trace, dtype)``
  -- Section 5.3's periodic boundary (both ends coupled), synchronous and
  asynchronous (trace uint8[K][S][2]: S boundaries on the ring).
* ``async_blocked(u0, r, c1, cN, S, q, T, K, trace, dtype)`` -- the bounded-delay
  model applied to blocks of T steps: segments exchange T-wide edge strips once
  per block, each strip up to q-1 blocks old (trace uint8[ceil(K/T)][S-1][2]).
* ``async_blocked_split(u0, r, c1, cN, offsets, q, T, K, trace, dtype)`` -- the same
  model on a given split of the rod into segments (S+1 offsets; every segment but
  the first and the last holds at least T points).
* ``async_blocked_periodic(u0, r, S, q, T, K, trace, dtype)`` -- the same model on
  the periodic ring of Section 5.3 (trace uint8[ceil(K/T)][S][2]).
* ``segments(N, S)`` -- the contiguous split of the N points into S segments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "heat1d_oracle.c"), os.path.join(_HERE, "heat1d_oracle_body.h")]
_LIB_PATH = os.path.join(_HERE, "libheat1d_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no vector extensions, no -march)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, i32, dbl, flt, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float, ctypes.c_void_p
        lib.oracle_segments.argtypes = [i64, i64, vp]
        lib.oracle_sync_f64.argtypes = [i64, dbl, dbl, dbl, vp, i64, vp]
        lib.oracle_sync_f32.argtypes = [i64, flt, flt, flt, vp, i64, vp]
        lib.oracle_async_f64.argtypes = [i64, dbl, dbl, dbl, i64, i32, vp, i64, vp, vp]
        lib.oracle_async_f32.argtypes = [i64, flt, flt, flt, i64, i32, vp, i64, vp, vp]
        lib.oracle_adjoint_f64.argtypes = [i64, dbl, dbl, dbl, i64, i32, vp, i64, vp, vp, vp, vp, vp]
        lib.oracle_sync_periodic_f64.argtypes = [i64, dbl, vp, i64, vp]
        lib.oracle_sync_periodic_f32.argtypes = [i64, flt, vp, i64, vp]
        lib.oracle_async_periodic_f64.argtypes = [i64, dbl, i64, i32, vp, i64, vp, vp]
        lib.oracle_async_periodic_f32.argtypes = [i64, flt, i64, i32, vp, i64, vp, vp]
        lib.oracle_async_blocked_f64.argtypes = [i64, dbl, dbl, dbl, i64, i32, i64, vp, i64, vp, vp]
        lib.oracle_async_blocked_f32.argtypes = [i64, flt, flt, flt, i64, i32, i64, vp, i64, vp, vp]
        lib.oracle_async_blocked_split_f64.argtypes = [i64, dbl, dbl, dbl, i64, vp, i32, i64, vp, i64, vp, vp]
        lib.oracle_async_blocked_split_f32.argtypes = [i64, flt, flt, flt, i64, vp, i32, i64, vp, i64, vp, vp]
        lib.oracle_async_blocked_periodic_f64.argtypes = [i64, dbl, i64, i32, i64, vp, i64, vp, vp]
        lib.oracle_async_blocked_periodic_f32.argtypes = [i64, flt, i64, i32, i64, vp, i64, vp, vp]
        for f in (lib.oracle_segments, lib.oracle_sync_f64, lib.oracle_sync_f32, lib.oracle_async_f64,
                  lib.oracle_async_f32, lib.oracle_adjoint_f64, lib.oracle_sync_periodic_f64,
                  lib.oracle_sync_periodic_f32, lib.oracle_async_periodic_f64, lib.oracle_async_periodic_f32,
                  lib.oracle_async_blocked_f64, lib.oracle_async_blocked_f32,
                  lib.oracle_async_blocked_split_f64, lib.oracle_async_blocked_split_f32,
                  lib.oracle_async_blocked_periodic_f64, lib.oracle_async_blocked_periodic_f32):
            f.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError("%s failed with status %d" % (what, rc))


def _np_dtype(dtype) -> np.dtype:
    dt = np.dtype(dtype)
    if dt not in (np.dtype(np.float64), np.dtype(np.float32)):
        raise ValueError("oracle dtype must be float64 or float32")
    return dt


def segments(N: int, S: int) -> np.ndarray:
    """Offsets (S+1 values) of the contiguous split of N points into S segments."""
    off = np.zeros(S + 1, dtype=np.int64)
    _check(_load().oracle_segments(N, S, _ptr(off)), "oracle_segments")
    return off


def sync(u0, r, c1, cN, K, dtype=np.float64) -> np.ndarray:
    """u(K) of the synchronous update (Eq. eqn:sync).  dtype=float32 runs the
    same expression in float with fmaf (r, c1, cN rounded to float)."""
    dt = _np_dtype(dtype)
    u0 = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(u0)
    lib = _load()
    fn = lib.oracle_sync_f64 if dt == np.float64 else lib.oracle_sync_f32
    _check(fn(u0.size, float(r), float(c1), float(cN), _ptr(u0), int(K), _ptr(out)), "oracle_sync")
    return out


def async_replay(u0, r, c1, cN, S, q, K, trace, dtype=np.float64) -> np.ndarray:
    """u(K) of the asynchronous update (Eq. eqn:async) driven by ``trace``
    (uint8, shape (K, S-1, 2) or flat; see heat1d_oracle.c for the layout)."""
    dt = _np_dtype(dtype)
    u0 = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(u0)
    tr = None
    if trace is not None:
        tr = np.ascontiguousarray(trace, dtype=np.uint8).reshape(-1)
        if tr.size != int(K) * (int(S) - 1) * 2:
            raise ValueError("trace has %d entries, expected K*(S-1)*2 = %d" % (tr.size, int(K) * (int(S) - 1) * 2))
    lib = _load()
    fn = lib.oracle_async_f64 if dt == np.float64 else lib.oracle_async_f32
    _check(fn(u0.size, float(r), float(c1), float(cN), int(S), int(q), _ptr(u0), int(K), _ptr(tr), _ptr(out)),
           "oracle_async")
    return out


def adjoint(u0, r, c1, cN, K, u_obs, S=1, q=1, trace=None):
    """FP64 (loss, grad_u0, grad_r) of L = 0.5*||u(K) - u_obs||^2.
    trace=None is the synchronous run."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    u_obs = np.ascontiguousarray(u_obs, dtype=np.float64)
    g = np.empty_like(u0)
    gr = ctypes.c_double(0.0)
    ls = ctypes.c_double(0.0)
    tr = None
    if trace is not None:
        tr = np.ascontiguousarray(trace, dtype=np.uint8).reshape(-1)
        if tr.size != int(K) * (int(S) - 1) * 2:
            raise ValueError("trace size mismatch")
    _check(_load().oracle_adjoint_f64(u0.size, float(r), float(c1), float(cN), int(S), int(q), _ptr(u0), int(K),
                                      _ptr(tr), _ptr(u_obs), _ptr(g), ctypes.byref(gr), ctypes.byref(ls)),
           "oracle_adjoint")
    return ls.value, g, gr.value


def sync_periodic(u0, r, K, dtype=np.float64) -> np.ndarray:
    """u(K) of the periodic synchronous update (Section 5.3)."""
    dt = _np_dtype(dtype)
    u0 = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(u0)
    lib = _load()
    fn = lib.oracle_sync_periodic_f64 if dt == np.float64 else lib.oracle_sync_periodic_f32
    _check(fn(u0.size, float(r), _ptr(u0), int(K), _ptr(out)), "oracle_sync_periodic")
    return out


def async_periodic(u0, r, S, q, K, trace, dtype=np.float64) -> np.ndarray:
    """u(K) of the periodic asynchronous update driven by ``trace``
    (uint8, shape (K, S, 2) or flat)."""
    dt = _np_dtype(dtype)
    u0 = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(u0)
    tr = np.ascontiguousarray(trace, dtype=np.uint8).reshape(-1)
    if tr.size != int(K) * int(S) * 2:
        raise ValueError("trace has %d entries, expected K*S*2 = %d" % (tr.size, int(K) * int(S) * 2))
    lib = _load()
    fn = lib.oracle_async_periodic_f64 if dt == np.float64 else lib.oracle_async_periodic_f32
    _check(fn(u0.size, float(r), int(S), int(q), _ptr(u0), int(K), _ptr(tr), _ptr(out)), "oracle_async_periodic")
    return out


def async_blocked(u0, r, c1, cN, S, q, T, K, trace, dtype=np.float64) -> np.ndarray:
    """u(K) of the asynchronous run with temporal blocking: blocks of T steps,
    T-wide halo strips taken up to q-1 blocks old (trace uint8, shape
    (ceil(K/T), S-1, 2) or flat; see heat1d_oracle_body.h for the definition)."""
    dt = _np_dtype(dtype)
    u0 = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(u0)
    nb = (int(K) + int(T) - 1) // int(T)
    tr = None
    if trace is not None:
        tr = np.ascontiguousarray(trace, dtype=np.uint8).reshape(-1)
        if tr.size != nb * (int(S) - 1) * 2:
            raise ValueError("trace has %d entries, expected ceil(K/T)*(S-1)*2 = %d" % (tr.size, nb * (int(S) - 1) * 2))
    lib = _load()
    fn = lib.oracle_async_blocked_f64 if dt == np.float64 else lib.oracle_async_blocked_f32
    _check(fn(u0.size, float(r), float(c1), float(cN), int(S), int(q), int(T), _ptr(u0), int(K), _ptr(tr), _ptr(out)),
           "oracle_async_blocked")
    return out


def async_blocked_split(u0, r, c1, cN, offsets, q, T, K, trace, dtype=np.float64) -> np.ndarray:
    """u(K) of the blocked asynchronous model on the segments given by
    ``offsets`` (S+1 int64 values from 0 to N); trace uint8, shape
    (ceil(K/T), S-1, 2) or flat."""
    dt = _np_dtype(dtype)
    u0 = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(u0)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    S = off.size - 1
    nb = (int(K) + int(T) - 1) // int(T)
    tr = None
    if trace is not None:
        tr = np.ascontiguousarray(trace, dtype=np.uint8).reshape(-1)
        if tr.size != nb * (S - 1) * 2:
            raise ValueError("trace has %d entries, expected ceil(K/T)*(S-1)*2 = %d" % (tr.size, nb * (S - 1) * 2))
    lib = _load()
    fn = lib.oracle_async_blocked_split_f64 if dt == np.float64 else lib.oracle_async_blocked_split_f32
    _check(fn(u0.size, float(r), float(c1), float(cN), S, _ptr(off), int(q), int(T), _ptr(u0), int(K), _ptr(tr),
              _ptr(out)), "oracle_async_blocked_split")
    return out


def async_blocked_periodic(u0, r, S, q, T, K, trace, dtype=np.float64) -> np.ndarray:
    """u(K) of the blocked asynchronous model on the periodic ring (Section
    5.3; trace uint8, shape (ceil(K/T), S, 2) or flat)."""
    dt = _np_dtype(dtype)
    u0 = np.ascontiguousarray(u0, dtype=dt)
    out = np.empty_like(u0)
    nb = (int(K) + int(T) - 1) // int(T)
    tr = np.ascontiguousarray(trace, dtype=np.uint8).reshape(-1)
    if tr.size != nb * int(S) * 2:
        raise ValueError("trace has %d entries, expected ceil(K/T)*S*2 = %d" % (tr.size, nb * int(S) * 2))
    lib = _load()
    fn = lib.oracle_async_blocked_periodic_f64 if dt == np.float64 else lib.oracle_async_blocked_periodic_f32
    _check(fn(u0.size, float(r), int(S), int(q), int(T), _ptr(u0), int(K), _ptr(tr), _ptr(out)),
           "oracle_async_blocked_periodic")
    return out

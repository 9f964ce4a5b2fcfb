"""Planted mistakes: each one, put into a copy of the oracle's C source on the
CPU, must make at least one pin fail.

The copy is compiled into a temporary directory and loaded with ctypes; the
oracle itself is never modified.  The mistakes are the plausible ones a
reading of the paper could make: a wrong neighbour, a wrong sign, a swapped
delay side, a delay taken from the wrong step or block, a halo one point too
narrow, a wrong wrap-around and a transposed adjoint scatter.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from paper_1510_08982_gb300 import inputs
from tests import pins

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_DIR = os.path.join(os.path.dirname(HERE), "oracle")

i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p


def _p(a):
    return None if a is None else a.ctypes.data_as(vp)


def build_mutant(tmp, func, old, new):
    """Copies the oracle sources, replaces the first `old` inside function
    `func` of the body by `new`, compiles and loads the copy."""
    for f in ("heat1d_oracle.c", "heat1d_oracle_body.h"):
        shutil.copy(os.path.join(ORACLE_DIR, f), os.path.join(tmp, f))
    for f in ("heat1d_oracle_body.h", "heat1d_oracle.c"):
        path = os.path.join(tmp, f)
        src = open(path).read()
        start = src.find(func + ")(") if f.endswith(".h") else src.find("int " + func + "(")
        if start < 0:
            continue
        at = src.find(old, start)
        assert at >= 0, "mutation text not found in %s" % func
        src = src[:at] + new + src[at + len(old):]
        open(path, "w").write(src)
        break
    else:
        raise AssertionError("function %s not found" % func)
    lib_path = os.path.join(tmp, "libmutant.so")
    subprocess.run(["gcc", "-std=c11", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o", lib_path,
                    os.path.join(tmp, "heat1d_oracle.c"), "-lm"], check=True)
    lib = ctypes.CDLL(lib_path)
    lib.oracle_sync_f64.argtypes = [i64, dbl, dbl, dbl, vp, i64, vp]
    lib.oracle_async_f64.argtypes = [i64, dbl, dbl, dbl, i64, i32, vp, i64, vp, vp]
    lib.oracle_async_blocked_f64.argtypes = [i64, dbl, dbl, dbl, i64, i32, i64, vp, i64, vp, vp]
    lib.oracle_sync_periodic_f64.argtypes = [i64, dbl, vp, i64, vp]
    lib.oracle_adjoint_f64.argtypes = [i64, dbl, dbl, dbl, i64, i32, vp, i64, vp, vp, vp, vp, vp]
    lib.oracle_async_blocked_periodic_f64.argtypes = [i64, dbl, i64, i32, i64, vp, i64, vp, vp]
    return lib


# Pin checks against a loaded library: each returns True when every pin holds.


def pins_sync(lib):
    rng = np.random.default_rng(0)
    N, K = 12, 10
    u0 = rng.integers(-16, 17, size=N) / 16.0
    out = np.empty(N)
    lib.oracle_sync_f64(N, 0.25, 0.5, -0.25, _p(u0), K, _p(out))
    return [Fraction(v) for v in out] == pins.brute_sync_fraction(u0, Fraction(1, 4), 0.5, -0.25, K)


def pins_async(lib):
    rng = np.random.default_rng(1)
    N, S, q, K = 12, 4, 3, 12
    u0 = rng.integers(-16, 17, size=N) / 16.0
    tr = rng.integers(0, q, size=(K, S - 1, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(K)[:, None, None]).astype(np.uint8)
    out = np.empty(N)
    lib.oracle_async_f64(N, 0.25, 0.25, -0.75, S, q, _p(u0), K, _p(tr), _p(out))
    return [Fraction(v) for v in out] == pins.brute_async_fraction(u0, Fraction(1, 4), 0.25, -0.75, S, q, trc)


def pins_blocked(lib):
    rng = np.random.default_rng(2)
    N, S, q, T, K = 16, 4, 3, 4, 12
    u0 = rng.integers(-16, 17, size=N) / 16.0
    nb = (K + T - 1) // T
    tr = rng.integers(0, q, size=(nb, S - 1, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(nb)[:, None, None]).astype(np.uint8)
    out = np.empty(N)
    lib.oracle_async_blocked_f64(N, 0.25, 0.25, -0.75, S, q, T, _p(u0), K, _p(tr), _p(out))
    ok = [Fraction(v) for v in out] == pins.brute_async_blocked_fraction(u0, Fraction(1, 4), 0.25, -0.75, S, q, T,
                                                                         K, trc)
    z = np.zeros_like(tr)
    ref = np.empty(N)
    lib.oracle_sync_f64(N, 0.25, 0.25, -0.75, _p(u0), K, _p(ref))
    lib.oracle_async_blocked_f64(N, 0.25, 0.25, -0.75, S, q, T, _p(u0), K, _p(z), _p(out))
    return ok and np.array_equal(out, ref)


def pins_blocked_periodic(lib):
    rng = np.random.default_rng(6)
    N, S, q, T, K = 15, 5, 3, 3, 10
    u0 = rng.integers(-16, 17, size=N) / 16.0
    nb = (K + T - 1) // T
    tr = rng.integers(0, q, size=(nb, S, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(nb)[:, None, None]).astype(np.uint8)
    out = np.empty(N)
    lib.oracle_async_blocked_periodic_f64(N, 0.25, S, q, T, _p(u0), K, _p(tr), _p(out))
    return [Fraction(v) for v in out] == pins.brute_async_blocked_periodic_fraction(u0, Fraction(1, 4), S, q, T, K,
                                                                                    trc)


def pins_periodic(lib):
    rng = np.random.default_rng(3)
    N, K = 10, 9
    u0 = rng.integers(-16, 17, size=N) / 16.0
    out = np.empty(N)
    lib.oracle_sync_periodic_f64(N, 0.25, _p(u0), K, _p(out))
    return [Fraction(v) for v in out] == pins.brute_sync_periodic_fraction(u0, Fraction(1, 4), K)


def pins_adjoint(lib):
    rng = np.random.default_rng(4)
    N, S, q, K = 10, 3, 3, 8
    u0 = rng.uniform(-1, 1, size=N)
    u_obs = rng.uniform(-1, 1, size=N)
    tr = rng.integers(0, q, size=(K, S - 1, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(K)[:, None, None]).astype(np.uint8)
    g = np.empty(N)
    gr, ls = ctypes.c_double(), ctypes.c_double()
    lib.oracle_adjoint_f64(N, 0.3, 0.1, -0.2, S, q, _p(u0), K, _p(tr), _p(u_obs), _p(g), ctypes.byref(gr),
                           ctypes.byref(ls))
    L, G, GR = pins.brute_adjoint_float(u0, Fraction(3, 10), 0.1, -0.2, S, q, trc, u_obs)
    return abs(ls.value - L) < 1e-12 and np.abs(g - G).max() < 1e-12 and abs(gr.value - GR) < 1e-11


MUTATIONS = [
    ("sync: right neighbour read twice", "oracle_sync", pins_sync,
     "(uR - (REAL)2 * u) + uL", "(uR - (REAL)2 * u) + uR"),
    ("sync: wrong sign of the centre term", "oracle_sync", pins_sync,
     "(uR - (REAL)2 * u)", "(uR + (REAL)2 * u)"),
    ("async: left read takes the right side's delay", "oracle_async", pins_async,
     "seg[i - 1]) * 2 + 1]", "seg[i - 1]) * 2 + 0]"),
    ("async: delay taken from the next step", "oracle_async", pins_async,
     "trace[(k * (S - 1) + seg[i]) * 2 + 0]", "trace[((k + 1 < K ? k + 1 : k) * (S - 1) + seg[i]) * 2 + 0]"),
    ("async: delayed read of the own point", "oracle_async", pins_async,
     "u = H(k, i)", "u = H(tL, i)"),
    ("blocked: left strip always current", "oracle_async_blocked_split", pins_blocked,
     "bl = b - (d < b ? d : b);", "bl = b;"),
    ("blocked: halo one point too narrow", "oracle_async_blocked_split", pins_blocked,
     "lo - T > 0 ? lo - T : 0", "lo - T + 1 > 0 ? lo - T + 1 : 0"),
    ("blocked: sides swapped", "oracle_async_blocked_split", pins_blocked,
     "(s - 1)) * 2 + 1]", "(s - 1)) * 2 + 0]"),
    ("blocked periodic: left halo with the right side's delay", "oracle_async_blocked_periodic",
     pins_blocked_periodic, "(s + S - 1) % S) * 2 + 1]", "(s + S - 1) % S) * 2 + 0]"),
    ("periodic: wrap-around to the wrong end", "oracle_sync_periodic", pins_periodic,
     "a[(i + N - 1) % N]", "a[(i + N - 2) % N]"),
    ("adjoint: scatter to the wrong time level", "oracle_adjoint_f64", pins_adjoint,
     "LL(tR, i + 1) += r * g;", "LL(tL, i + 1) += r * g;"),
    ("adjoint: r-gradient sign", "oracle_adjoint_f64", pins_adjoint,
     "double du = (UU(tR, i + 1) - 2.0 * UU(k, i))", "double du = (UU(tR, i + 1) + 2.0 * UU(k, i))"),
]


@pytest.mark.parametrize("name,func,check,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, func, check, old, new):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    unmutated = build_mutant(str(tmp_path), func, old, old)
    assert check(unmutated), "pins must hold for the unmodified oracle"
    d = tmp_path / "m"
    d.mkdir()
    mutant = build_mutant(str(d), func, old, new)
    assert not check(mutant), "planted mistake '%s' passed every pin" % name

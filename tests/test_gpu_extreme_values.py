"""GPU parity on values that reach the corners of IEEE 754 arithmetic in the
update: operands spread over the whole exponent range (subnormals among
them), signed zeros, sums that overflow to infinity, and infinite and NaN
states.  Every on-chip and streamed run of the library -- synchronous,
asynchronous replay, blocked replay, streamed and batched -- against the
oracle, bit for bit (a NaN matches any NaN: IEEE 754 leaves payloads open).

The update is r*((uR - 2u) + uL) + u with uR - 2u formed by one fused
multiply-add (Section 4's order).  The oracle forms 2u first, so the two agree
while 2u is finite: every finite state here is below 2^1023 in magnitude
(2^127 in FP32); larger values appear only as infinities.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch  # noqa: F401
    from paper_1510_08982_gb300 import build, heat1d
    build.build()
    return heat1d


def same_bits(a, b):
    a = np.asarray(a)
    b = np.asarray(b, dtype=a.dtype)
    ut = np.uint64 if a.dtype == np.float64 else np.uint32
    return bool(np.all((np.isnan(a) & np.isnan(b)) | (a.view(ut) == b.view(ut))))


def states(kind, N, dtype, seed):
    rng = np.random.default_rng(seed)
    lo, hi = (-1074, 1000) if dtype == "float64" else (-149, 100)
    sign = np.where(rng.random(N) < 0.5, -1.0, 1.0)
    if kind == "wide":  # every exponent, subnormals included, and some signed zeros
        u = sign * np.ldexp(1.0 + rng.random(N), rng.integers(lo, hi, size=N))
        u[rng.random(N) < 0.05] = 0.0
        u[rng.random(N) < 0.05] = -0.0
    elif kind == "tiny":  # subnormals and zeros only: exact sums, signs of zero
        u = sign * np.ldexp(rng.integers(0, 8, size=N).astype(np.float64), lo)
    elif kind == "huge":  # |u| in [2^1020, 2^1022) (2^124..2^126 in FP32): large exponents, no overflow
        u = sign * np.ldexp(1.0 + rng.random(N), rng.integers(1020, 1022, size=N) if dtype == "float64"
                            else rng.integers(124, 126, size=N))
    elif kind == "overflow":  # A, 0, A, 0, ... with A = 1.5 * 2^1023: uL + uR overflows at the zeros
        A = 1.5 * 2.0 ** (1023 if dtype == "float64" else 127)
        u = np.where(np.arange(N) % 2 == 0, sign * A, 0.0)
    else:  # "special": smooth data with infinities and NaNs planted
        u = np.sin(np.linspace(0.0, 9.0, N))
        idx = rng.choice(N, size=6, replace=False)
        u[idx] = [np.inf, -np.inf, np.nan, np.inf, -np.inf, np.nan]
    return u.astype(np.float32 if dtype == "float32" else np.float64)


KINDS = ["wide", "tiny", "huge", "overflow", "special"]
N, S, Q, T = 3001, 8, 3, 16


def steps(kind):
    return 1 if kind == "overflow" else 300  # one step of overflow leaves infinities of both signs


def ends(kind, dtype):
    if kind == "tiny":
        return -0.0, 0.0
    if kind in ("huge", "overflow"):
        return (2.0 ** 1021, -(2.0 ** 1021)) if dtype == "float64" else (2.0 ** 125, -(2.0 ** 125))
    return 0.75, -1.25


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("kind", KINDS)
def test_extreme_on_chip_runs(H, dtype, kind):
    npdt = np.float32 if dtype == "float32" else np.float64
    u0 = states(kind, N, dtype, seed=KINDS.index(kind))
    c1, cN = ends(kind, dtype)
    r, K = 0.375, steps(kind)
    with H.Heat1d(N, r, c1, cN, dtype=dtype, segments=S, q=Q, halo_steps=T, sync_mode=1) as h:
        h.set_u(u0)
        h.run_sync(K)
        h.sync()
        assert same_bits(h.get_u(device=False), oracle.sync(u0, r, c1, cN, K, dtype=npdt)), "sync"
        tr = inputs.delay_trace(K, S, Q, seed=3)
        h.set_u(u0)
        h.replay(K, tr)
        h.sync()
        assert same_bits(h.get_u(device=False), oracle.async_replay(u0, r, c1, cN, S, Q, K, tr, dtype=npdt)), \
            "replay"
        btr = inputs.delay_trace((K + T - 1) // T, S, Q, seed=4)
        h.set_u(u0)
        h.replay_blocked(K, btr)
        h.sync()
        assert same_bits(h.get_u(device=False), oracle.async_blocked(u0, r, c1, cN, S, Q, T, K, btr, dtype=npdt)), \
            "blocked"


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("kind", KINDS)
def test_extreme_streamed_and_batched(H, dtype, kind):
    import torch
    npdt = np.float32 if dtype == "float32" else np.float64
    u0 = states(kind, N, dtype, seed=10 + KINDS.index(kind))
    c1, cN = ends(kind, dtype)
    r, K = 0.5, steps(kind)
    ref = oracle.sync(u0, r, c1, cN, K, dtype=npdt)
    with H.Heat1d(N, r, c1, cN, dtype=dtype, sync_mode=2, halo_steps=T, block_threads=64) as h:
        h.set_u(u0)
        h.run_sync(K)
        h.sync()
        assert same_bits(h.get_u(device=False), ref), "streamed"
    off, total = H.pack_offsets([N, N])
    u = np.zeros(total, dtype=npdt)
    u[off[0]:off[0] + N] = u0
    u[off[1]:off[1] + N] = u0[::-1]
    specs = [(int(off[0]), N, K, r, c1, cN), (int(off[1]), N, max(1, K // 2), r, c1, cN)]
    ut = torch.tensor(u, device="cuda")
    with H.Batch(specs, dtype=dtype, elems_per_thread=4, block_threads=64, halo_steps=8) as b:
        b.run(ut)
        b.sync()
    got = ut.cpu().numpy()
    assert same_bits(got[off[0]:off[0] + N], ref), "batched"
    assert same_bits(got[off[1]:off[1] + N], oracle.sync(u0[::-1].copy(), r, c1, cN, max(1, K // 2), dtype=npdt)), \
        "batched 2"

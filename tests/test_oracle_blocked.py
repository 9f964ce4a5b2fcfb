"""Pins of the oracle's asynchronous run with temporal blocking.

The model (blocks of T steps; each segment advances a block on its own points
plus T-wide halo strips taken from its neighbours up to q-1 blocks old) is
defined in oracle/heat1d_oracle_body.h.  It is checked here against what fixes
it independently: the synchronous run (all delays 0), Eq. (eqn:async) (T = 1),
an exact rational restatement as whole-vector matrix powers (tests/pins.py),
the maximum principle and the unique steady state.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs
from tests import pins


def nblocks(K, T):
    return (K + T - 1) // T


@pytest.mark.parametrize("T,K", [(1, 300), (4, 300), (7, 300), (64, 1000), (128, 1000), (5, 3)])
def test_blocked_zero_trace_equals_sync_bitwise(T, K):
    """All strips current (d = 0) is the synchronous run, bit for bit, in both
    precisions and for a ragged last block."""
    rod = inputs.small_rod(K=K)
    tr = np.zeros((nblocks(K, T), 7, 2), dtype=np.uint8)
    for dt in (np.float64, np.float32):
        a = oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, T, K, tr, dtype=dt)
        b = oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, K, dtype=dt)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_blocked_T1_is_eqn_async(seed):
    """Blocks of one step are Eq. (eqn:async) with the same trace."""
    rod = inputs.small_rod(K=500)
    tr = inputs.delay_trace(rod.K, 8, 3, seed=seed)
    for dt in (np.float64, np.float32):
        a = oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, 1, rod.K, tr, dtype=dt)
        b = oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, rod.K, tr, dtype=dt)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("N,S,q,T,K,seed", [(12, 3, 2, 2, 9, 0), (13, 3, 3, 3, 11, 1), (16, 4, 3, 4, 12, 2),
                                            (10, 2, 4, 5, 14, 3), (15, 5, 2, 3, 10, 4), (9, 3, 1, 3, 7, 5)])
def test_blocked_brute_force_exact(N, S, q, T, K, seed):
    """Exact rational whole-vector matrix powers against the oracle bit for bit
    (dyadic data, r = 1/4)."""
    rng = np.random.default_rng(seed)
    u0 = rng.integers(-16, 17, size=N) / 16.0
    nb = nblocks(K, T)
    tr = rng.integers(0, q, size=(nb, S - 1, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(nb)[:, None, None]).astype(np.uint8)
    exact = pins.brute_async_blocked_fraction(u0, Fraction(1, 4), 0.25, -0.75, S, q, T, K, trc)
    got = oracle.async_blocked(u0, 0.25, 0.25, -0.75, S, q, T, K, tr)
    assert [Fraction(v) for v in got] == exact


def test_blocked_stale_strip_and_sides_matter():
    """One stale strip changes the result, and swapping the trace's sides
    changes it again: the brute-force pin would see a side or block mix-up."""
    rng = np.random.default_rng(5)
    N, S, q, T, K = 24, 3, 3, 4, 24
    u0 = rng.integers(-16, 17, size=N) / 16.0
    nb = nblocks(K, T)
    z = np.zeros((nb, S - 1, 2), dtype=np.uint8)
    tr = z.copy()
    tr[3, 0, 0] = 2
    tr[4, 1, 1] = 1
    base = oracle.async_blocked(u0, 0.25, 0.0, 0.0, S, q, T, K, z)
    a = oracle.async_blocked(u0, 0.25, 0.0, 0.0, S, q, T, K, tr)
    b = oracle.async_blocked(u0, 0.25, 0.0, 0.0, S, q, T, K, tr[:, :, ::-1].copy())
    assert not np.array_equal(a, base) and not np.array_equal(a, b)


@pytest.mark.parametrize("r", [0.1, 0.5])
def test_blocked_maximum_principle(r):
    rng = np.random.default_rng(4)
    N, S, q, T, K = 300, 6, 3, 16, 400
    u0 = rng.uniform(-1, 1, size=N)
    tr = inputs.delay_trace(nblocks(K, T), S, q, seed=7)
    u = oracle.async_blocked(u0, r, 0.2, -0.3, S, q, T, K, tr)
    lo, hi = min(u0[1:-1].min(), 0.2, -0.3), max(u0[1:-1].max(), 0.2, -0.3)
    assert u.min() >= lo - 1e-13 and u.max() <= hi + 1e-13


def test_blocked_unique_steady_state():
    """With Dirichlet ends the blocked asynchronous run reaches the linear
    steady state whatever the (bounded) strip delays."""
    N, S, q, T, K = 24, 3, 3, 4, 30000
    u0 = inputs.paper_rod(N=N).u0
    x = inputs.grid_x(N)
    for seed in (0, 1):
        tr = inputs.delay_trace(nblocks(K, T), S, q, seed=seed)
        u = oracle.async_blocked(u0, 0.5, 1.0, 0.0, S, q, T, K, tr)
        assert np.abs(u - (1.0 - x)).max() < 1e-12


def test_blocked_rejects_bad_arguments():
    rod = inputs.small_rod(K=10)
    tr = np.zeros((nblocks(10, 4), 7, 2), dtype=np.uint8)
    tr[1, 2, 1] = 3
    with pytest.raises(oracle.OracleError):  # delay outside the window
        oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, 4, 10, tr)
    with pytest.raises(oracle.OracleError):  # halo wider than the shortest segment (128 points)
        oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, 129, 10, np.zeros((1, 7, 2), np.uint8))
    with pytest.raises(ValueError):
        oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, 4, 10, np.zeros((2, 7, 2), np.uint8))


# ----------------------------------------------------------------------------- periodic ring (Section 5.3)


@pytest.mark.parametrize("T,K", [(1, 200), (5, 200), (16, 333)])
def test_blocked_periodic_zero_trace_is_periodic_sync(T, K):
    rng = np.random.default_rng(T)
    u0 = rng.uniform(-1, 1, size=300)
    tr = np.zeros((nblocks(K, T), 6, 2), dtype=np.uint8)
    for dt in (np.float64, np.float32):
        a = oracle.async_blocked_periodic(u0, 0.4, 6, 3, T, K, tr, dtype=dt)
        assert np.array_equal(a, oracle.sync_periodic(u0, 0.4, K, dtype=dt))


def test_blocked_periodic_T1_is_periodic_async():
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1, 1, size=301)
    tr = inputs.periodic_delay_trace(250, 7, 3, seed=4)
    a = oracle.async_blocked_periodic(u0, 0.45, 7, 3, 1, 250, tr)
    assert np.array_equal(a, oracle.async_periodic(u0, 0.45, 7, 3, 250, tr))


@pytest.mark.parametrize("N,S,q,T,K,seed", [(12, 3, 3, 2, 9, 0), (14, 2, 2, 3, 13, 1), (15, 5, 3, 3, 10, 2)])
def test_blocked_periodic_brute_force_exact(N, S, q, T, K, seed):
    """Exact rational restatement, on shapes whose two halos do not share a
    point (2T at most the neighbours' length): the whole-vector form holds
    one value per point, the tile one copy per strip."""
    rng = np.random.default_rng(seed)
    u0 = rng.integers(-16, 17, size=N) / 16.0
    nb = nblocks(K, T)
    tr = rng.integers(0, q, size=(nb, S, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(nb)[:, None, None]).astype(np.uint8)
    exact = pins.brute_async_blocked_periodic_fraction(u0, Fraction(1, 4), S, q, T, K, trc)
    got = oracle.async_blocked_periodic(u0, 0.25, S, q, T, K, tr)
    assert [Fraction(v) for v in got] == exact


def test_blocked_periodic_sum_drifts_only_with_delays():
    """The circulant update conserves the sum; stale strips break that (the
    'no unique steady state' of Section 5.3), while current ones keep it up to
    rounding."""
    rng = np.random.default_rng(8)
    u0 = rng.uniform(0, 1, size=200)
    K, T, S, q = 400, 8, 5, 3
    z = np.zeros((nblocks(K, T), S, 2), dtype=np.uint8)
    assert abs(oracle.async_blocked_periodic(u0, 0.5, S, q, T, K, z).sum() - u0.sum()) < 1e-10
    tr = inputs.periodic_delay_trace(nblocks(K, T), S, q, seed=1)
    assert abs(oracle.async_blocked_periodic(u0, 0.5, S, q, T, K, tr).sum() - u0.sum()) > 1e-6


# --------------------------------------------------------------------------- given splits


def random_split(rng, N, S, T):
    """S+1 offsets with every segment but the first and the last >= T points;
    the first and the last may be shorter (down to one point)."""
    while True:
        inner = rng.integers(T, T + 6, size=S - 2) if S > 2 else np.zeros(0, dtype=np.int64)
        ends = rng.integers(1, T + 4, size=2)
        lens = np.concatenate([[ends[0]], inner, [ends[1]]]) if S > 1 else np.array([N])
        if lens.sum() == N:
            return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        if S > 1:
            lens[1 if S > 2 else 0] += N - lens.sum()
            if lens.min() >= 1 and (S <= 2 or lens[1:-1].min() >= T):
                return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


def test_split_with_the_standard_offsets_is_the_standard_model():
    rod = inputs.small_rod(K=400)
    tr = inputs.delay_trace(nblocks(400, 16), 8, 3, seed=7)
    a = oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, 16, 400, tr)
    b = oracle.async_blocked_split(rod.u0, rod.r, rod.c1, rod.cN, oracle.segments(1024, 8), 3, 16, 400, tr)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_split_zero_trace_equals_sync_bitwise(seed):
    """Any split with all strips current is the synchronous run, also with a
    first or last segment shorter than T."""
    rng = np.random.default_rng(seed)
    T, S = int(rng.integers(2, 9)), int(rng.integers(2, 7))
    N = int(T * S + rng.integers(3, 20))
    off = random_split(rng, N, S, T)
    K = int(rng.integers(5, 60))
    u0 = rng.uniform(-1, 1, size=N)
    tr = np.zeros((nblocks(K, T), S - 1, 2), dtype=np.uint8)
    for dt in (np.float64, np.float32):
        a = oracle.async_blocked_split(u0, 0.3, 0.5, -0.25, off, 3, T, K, tr, dtype=dt)
        assert np.array_equal(a, oracle.sync(u0, 0.3, 0.5, -0.25, K, dtype=dt))


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5])
def test_split_brute_force_exact(seed):
    """Exact rational whole-vector matrix powers on a random split (first and
    last segments may be shorter than T) against the oracle bit for bit
    (dyadic data, r = 1/4)."""
    rng = np.random.default_rng(100 + seed)
    T, S, q = int(rng.integers(2, 5)), int(rng.integers(2, 5)), int(rng.integers(1, 4))
    N = int(T * S + rng.integers(2, 6))
    off = random_split(rng, N, S, T)
    K = int(rng.integers(4, 13))
    u0 = rng.integers(-16, 17, size=N) / 16.0
    nb = nblocks(K, T)
    tr = rng.integers(0, q, size=(nb, S - 1, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(nb)[:, None, None]).astype(np.uint8)
    exact = pins.brute_async_blocked_fraction(u0, Fraction(1, 4), 0.25, -0.75, S, q, T, K, trc, offsets=off)
    got = oracle.async_blocked_split(u0, 0.25, 0.25, -0.75, off, q, T, K, tr)
    assert [Fraction(float(x)) for x in got] == exact


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_split_T1_is_the_switched_system(seed):
    """Blocks of one step on a given split are Eq. (eqn:async) on that split:
    exact rational brute force of the augmented switched system."""
    rng = np.random.default_rng(200 + seed)
    S, q = int(rng.integers(2, 5)), int(rng.integers(1, 4))
    N = int(S + rng.integers(3, 8))
    off = random_split(rng, N, S, 1)
    K = int(rng.integers(4, 11))
    u0 = rng.integers(-16, 17, size=N) / 16.0
    tr = rng.integers(0, q, size=(K, S - 1, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(K)[:, None, None]).astype(np.uint8)
    exact = pins.brute_async_fraction(u0, Fraction(1, 4), 0.25, -0.75, S, q, trc, offsets=off)
    got = oracle.async_blocked_split(u0, 0.25, 0.25, -0.75, off, q, 1, K, tr)
    assert [Fraction(float(x)) for x in got] == exact


def test_split_rejects_bad_offsets():
    u0 = np.zeros(20)
    tr = np.zeros((2, 2, 2), dtype=np.uint8)
    with pytest.raises(oracle.OracleError):   # an inner segment shorter than T
        oracle.async_blocked_split(u0, 0.25, 0, 0, np.array([0, 9, 11, 20]), 2, 4, 8, tr)
    with pytest.raises(oracle.OracleError):   # offsets not ending at N
        oracle.async_blocked_split(u0, 0.25, 0, 0, np.array([0, 9, 14, 19]), 2, 4, 8, tr)
    with pytest.raises(oracle.OracleError):   # an empty segment
        oracle.async_blocked_split(u0, 0.25, 0, 0, np.array([0, 9, 9, 20]), 2, 4, 8, tr)

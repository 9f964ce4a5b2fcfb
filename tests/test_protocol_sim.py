"""The exchange protocol of the asynchronous run (Section 3, Eq. (eqn:async)),
played by CPU threads (tests/protocol_sim.py): bounded delays, version rings
that are never read after being overwritten, flow control, replay from a
recorded trace, and failure by timeout.  The same for the blocked model
(strips of T points once per block) on uneven segments, as the blocked
kernel's segments and the batched launch's rod parts exchange them.  The
oracle replays every recorded trace."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from tests.protocol_sim import AsyncProtocol


def rod(N, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, size=N)


@pytest.mark.parametrize("S,q,seed", [(4, 1, 0), (4, 3, 1), (6, 2, 2), (5, 4, 3), (8, 3, 4)])
def test_free_run_is_a_run_of_eqn_async(S, q, seed):
    N, K, r = 61, 150, 0.37
    u0 = rod(N, seed)
    p = AsyncProtocol(u0, r, 0.25, -0.5, S, q, K, jitter_s=3e-4, seed=seed)
    assert p.run() == "ok"
    tr = p.trace
    assert tr.max(initial=0) < q
    assert all(int(tr[k].max(initial=0)) <= k for k in range(K))
    assert p.max_lead <= q  # flow control: no segment more than q versions ahead of a neighbour
    ref = oracle.async_replay(u0, r, 0.25, -0.5, S, q, K, tr)
    assert np.abs(p.u - ref).max() <= 1e-13  # unfused arithmetic against the oracle's fused one
    # the same trace replayed by the protocol gives the same state, bit for bit
    rep = AsyncProtocol(u0, r, 0.25, -0.5, S, q, K, trace=tr, jitter_s=3e-4, seed=seed + 100)
    assert rep.run() == "ok"
    assert np.array_equal(rep.u, p.u)
    assert np.array_equal(rep.trace, tr)


def test_delays_occur_under_jitter():
    u0 = rod(40, 9)
    p = AsyncProtocol(u0, 0.3, 0.0, 0.0, 8, 3, 200, jitter_s=1e-3, seed=9)
    assert p.run() == "ok"
    hist = np.bincount(p.trace.reshape(-1), minlength=3)
    assert hist[1] + hist[2] > 0  # some reads were late
    ref = oracle.async_replay(u0, 0.3, 0.0, 0.0, 8, 3, 200, p.trace)
    assert np.abs(p.u - ref).max() <= 1e-13


def test_stalled_segment_times_out():
    u0 = rod(30, 5)
    t0 = time.monotonic()
    p = AsyncProtocol(u0, 0.3, 0.0, 0.0, 3, 2, 100, stall=1, limit_s=0.2, jitter_s=0)
    assert p.run() == "timeout"
    assert time.monotonic() - t0 < 10


def test_bad_trace_entry_is_rejected():
    u0 = rod(30, 6)
    tr = np.zeros((50, 2, 2), dtype=np.uint8)
    tr[20, 1, 0] = 2
    p = AsyncProtocol(u0, 0.3, 0.0, 0.0, 3, 2, 50, trace=tr, jitter_s=0)
    assert p.run() == "trace"


# ---------------------------------------------------------------- blocked model

from tests.protocol_sim import BlockedProtocol  # noqa: E402


def split_offsets(N, P):
    """Parts as the batched planner cuts a rod: P parts of N // P points, the
    first N % P one longer."""
    base, extra = divmod(N, P)
    off = [0]
    for p in range(P):
        off.append(off[-1] + base + (1 if p < extra else 0))
    return off


@pytest.mark.parametrize("offs,q,T,seed", [
    (split_offsets(73, 4), 3, 5, 0),
    (split_offsets(90, 6), 2, 8, 1),
    ([0, 3, 20, 41, 57, 60], 3, 4, 2),  # first and last segments shorter than T
    (split_offsets(64, 3), 1, 6, 3),    # q = 1: no delay at all
    (split_offsets(100, 5), 4, 3, 4),
])
def test_blocked_free_run_is_a_run_of_the_blocked_model(offs, q, T, seed):
    N, K, r = offs[-1], 157, 0.41
    u0 = rod(N, 40 + seed)
    p = BlockedProtocol(u0, r, 0.5, -0.25, offs, q, T, K, jitter_s=3e-4, seed=seed)
    assert p.run() == "ok"
    tr = p.trace
    assert tr.max(initial=0) < q
    assert all(int(tr[b].max(initial=0)) <= b for b in range(tr.shape[0]))
    assert p.max_lead <= q  # flow control: no segment more than q blocks ahead of a neighbour
    ref = oracle.async_blocked_split(u0, r, 0.5, -0.25, np.array(offs, dtype=np.int64), q, T, K, tr)
    assert np.abs(p.u - ref).max() <= 1e-13  # unfused arithmetic against the oracle's fused one
    rep = BlockedProtocol(u0, r, 0.5, -0.25, offs, q, T, K, trace=tr, jitter_s=3e-4, seed=seed + 100)
    assert rep.run() == "ok"
    assert np.array_equal(rep.u, p.u)
    assert np.array_equal(rep.trace, tr)


def test_blocked_delays_occur_under_jitter():
    offs = split_offsets(96, 8)
    u0 = rod(96, 50)
    p = BlockedProtocol(u0, 0.3, 0.0, 0.0, offs, 3, 4, 240, jitter_s=1e-3, seed=5)
    assert p.run() == "ok"
    hist = np.bincount(p.trace.reshape(-1), minlength=3)
    assert hist[1] + hist[2] > 0  # some strips were a block or two old
    ref = oracle.async_blocked_split(u0, 0.3, 0.0, 0.0, np.array(offs, dtype=np.int64), 3, 4, 240, p.trace)
    assert np.abs(p.u - ref).max() <= 1e-13


def test_blocked_with_one_step_blocks_is_the_step_model():
    """With T = 1 a block is a step and a strip is one edge value: a replay of
    the same delays through both simulators gives the same state."""
    N, S, q, K = 48, 6, 3, 120
    u0 = rod(N, 51)
    tr = np.random.default_rng(7).integers(0, q, size=(K, S - 1, 2)).astype(np.uint8)
    b = BlockedProtocol(u0, 0.35, 0.1, 0.2, split_offsets(N, S), q, 1, K, trace=tr, jitter_s=1e-4, seed=1)
    a = AsyncProtocol(u0, 0.35, 0.1, 0.2, S, q, K, trace=tr, jitter_s=1e-4, seed=2)
    assert b.run() == "ok" and a.run() == "ok"
    assert np.array_equal(b.u, a.u)


def test_blocked_stalled_segment_times_out():
    t0 = time.monotonic()
    p = BlockedProtocol(rod(40, 52), 0.3, 0.0, 0.0, split_offsets(40, 4), 2, 3, 90, stall=2, limit_s=0.2, jitter_s=0)
    assert p.run() == "timeout"
    assert time.monotonic() - t0 < 10


def test_blocked_bad_trace_entry_is_rejected():
    offs = split_offsets(40, 4)
    nb = (60 + 3 - 1) // 3
    tr = np.zeros((nb, 3, 2), dtype=np.uint8)
    tr[7, 2, 1] = 2
    p = BlockedProtocol(rod(40, 53), 0.3, 0.0, 0.0, offs, 2, 3, 60, trace=tr, jitter_s=0)
    assert p.run() == "trace"


@pytest.mark.parametrize("N,S,q,T,seed", [(64, 4, 3, 5, 0), (50, 2, 2, 7, 1), (90, 6, 4, 3, 2)])
def test_blocked_periodic_free_run_is_a_run_of_the_ring_model(N, S, q, T, seed):
    """The ring of Section 5.3 (S = 2: both halos from the one neighbour)."""
    from tests.protocol_sim import segment_offsets
    K, r = 140, 0.5
    u0 = rod(N, 60 + seed)
    p = BlockedProtocol(u0, r, 0.0, 0.0, segment_offsets(N, S), q, T, K, jitter_s=3e-4, seed=seed, periodic=True)
    assert p.run() == "ok"
    tr = p.trace
    assert tr.shape == ((K + T - 1) // T, S, 2) and tr.max(initial=0) < q
    ref = oracle.async_blocked_periodic(u0, r, S, q, T, K, tr)
    assert np.abs(p.u - ref).max() <= 1e-13
    rep = BlockedProtocol(u0, r, 0.0, 0.0, segment_offsets(N, S), q, T, K, trace=tr, jitter_s=3e-4, seed=seed + 7,
                          periodic=True)
    assert rep.run() == "ok"
    assert np.array_equal(rep.u, p.u)

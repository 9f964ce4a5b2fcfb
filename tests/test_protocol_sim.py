"""The exchange protocol of the asynchronous run (Section 3, Eq. (eqn:async)),
played by CPU threads (tests/protocol_sim.py): bounded delays, version rings
that are never read after being overwritten, flow control, replay from a
recorded trace, and failure by timeout.  The oracle replays every recorded
trace."""
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

"""GPU parity of the asynchronous run with temporal blocking (strips of T edge
points exchanged once per block of T steps, up to q-1 blocks old) against the
oracle, bit for bit: free runs through their recorded traces, replays of
seeded traces, the two reductions (all delays 0 = synchronous run; T = 1 =
Eq. (eqn:async)) and the failure paths."""
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


def nblocks(K, T):
    return (K + T - 1) // T


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,S,q,T,K", [(1024, 8, 3, 16, 1000), (1024, 8, 3, 64, 10000), (4099, 7, 2, 5, 777),
                                       (300, 100, 3, 1, 500), (2000, 3, 4, 100, 1234), (5000, 1, 3, 64, 300)])
def test_blocked_free_run_replays_in_oracle(H, dtype, N, S, q, T, K):
    """A free-running blocked run equals the oracle's blocked model driven by
    the trace the GPU recorded; the GPU replay of that trace gives the same
    state again."""
    npdt = np.float32 if dtype == "float32" else np.float64
    rod = inputs.small_rod(N=N, K=K)
    with H.Heat1d(N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q, halo_steps=T) as h:
        assert h.get_opts()["halo_steps"] == T
        tr = h.new_blocked_trace(K)
        assert tuple(tr.shape) == (nblocks(K, T), max(S - 1, 0), 2)
        h.set_u(rod.u0)
        h.run_async_blocked(K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
        if S > 1:
            assert trh.max() < q
            assert not trh[0].any()  # block 0 has only version 0
            assert np.all(trh <= np.arange(trh.shape[0])[:, None, None])
        assert np.array_equal(got, oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, S, q, T, K,
                                                        trh if S > 1 else None, dtype=npdt))
        h.set_u(rod.u0)
        h.replay_blocked(K, tr)
        h.sync()
        assert np.array_equal(h.get_u(device=False), got)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,S,q,T,K,seed", [(1024, 8, 3, 16, 1000, 0), (4099, 7, 3, 33, 2000, 1),
                                            (3000, 24, 2, 8, 901, 2), (700, 5, 5, 128, 1000, 3)])
def test_blocked_seeded_replay_bitwise(H, dtype, N, S, q, T, K, seed):
    npdt = np.float32 if dtype == "float32" else np.float64
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-1, 1, size=N)
    tr = inputs.delay_trace(nblocks(K, T), S, q, seed=seed)
    with H.Heat1d(N, 0.45, 0.3, -0.2, dtype=dtype, segments=S, q=q, halo_steps=T) as h:
        h.set_u(u0)
        h.replay_blocked(K, tr)  # host trace
        h.sync()
        got = h.get_u(device=False)
    assert np.array_equal(got, oracle.async_blocked(u0, 0.45, 0.3, -0.2, S, q, T, K, tr, dtype=npdt))


def test_blocked_zero_delays_is_the_synchronous_run(H):
    rod = inputs.small_rod(K=3000)
    T = 64
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, halo_steps=T) as h:
        h.set_u(rod.u0)
        h.replay_blocked(rod.K, np.zeros((nblocks(rod.K, T), 7, 2), dtype=np.uint8))
        h.sync()
        blocked = h.get_u(device=False)
        h.set_u(rod.u0)
        h.run_sync(rod.K)
        h.sync()
        sync = h.get_u(device=False)
    assert np.array_equal(blocked, sync)
    assert np.array_equal(sync, oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K))


def test_blocked_T1_is_eqn_async(H):
    """Blocks of one step replay Eq. (eqn:async): the same trace through the
    oracle's per-step asynchronous model gives the same state."""
    rod = inputs.small_rod(K=1500)
    tr = inputs.delay_trace(rod.K, 8, 3, seed=11)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, halo_steps=1) as h:
        h.set_u(rod.u0)
        h.replay_blocked(rod.K, tr)
        h.sync()
        got = h.get_u(device=False)
    assert np.array_equal(got, oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, rod.K, tr))


def test_blocked_full_size_rod(H):
    """The 2^20-point sine-mode rod, one segment per SM, T = 64, q = 3: the free
    run against the oracle through its trace (K = 640, ten blocks)."""
    import torch
    rod = inputs.sine_mode_rod(K=640)
    S = torch.cuda.get_device_properties(0).multi_processor_count
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=S, q=3, halo_steps=64) as h:
        h.set_u(rod.u0)
        tr = h.new_blocked_trace(rod.K)
        h.run_async_blocked(rod.K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
    assert np.array_equal(got, oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, S, 3, 64, rod.K, trh))


def test_blocked_snapshots_follow_the_run(H):
    """Snapshots of a blocked replay are the oracle's blocked states at those steps."""
    import torch
    rod = inputs.small_rod(K=512)
    T, every = 16, 64
    tr = inputs.delay_trace(nblocks(rod.K, T), 8, 3, seed=5)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, halo_steps=T) as h:
        snaps = torch.empty((rod.K // every + 1, rod.N), dtype=torch.float64, device="cuda")
        h.set_snapshots(snaps, every=every)
        h.set_u(rod.u0)
        h.replay_blocked(rod.K, tr)
        h.sync()
        h.set_snapshots(None)
        got = snaps.cpu().numpy()
    for row in (0, 3, rod.K // every):
        k = row * every
        ref = oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, T, k, tr[:nblocks(k, T)])
        assert np.array_equal(got[row], ref)


def test_blocked_rejects_bad_trace_and_periodic(H):
    rod = inputs.small_rod(K=100)
    tr = np.zeros((nblocks(100, 16), 7, 2), dtype=np.uint8)
    tr[3, 2, 0] = 3
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, halo_steps=16) as h:
        h.set_u(rod.u0)
        h.replay_blocked(100, tr)
        with pytest.raises(H.Heat1dError) as ei:
            h.sync()
        assert ei.value.code == H.ERR_TRACE
        h.set_u(rod.u0)  # the handle stays usable
        h.run_sync(10)
        h.sync()
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=1, q=3, boundary=1) as h:
        h.set_u(rod.u0)
        with pytest.raises(H.Heat1dError):  # a ring needs two segments
            h.run_async_blocked(10)


def test_blocked_stalled_segment_times_out(H):
    """A segment that never publishes (a flag nothing sets) makes its
    neighbours' bounded waits run out; the run reports a timeout and the
    context stays usable."""
    rod = inputs.small_rod(K=1000)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, halo_steps=16, stall_segment=3,
                  spin_limit_ns=200_000_000) as h:
        h.set_u(rod.u0)
        h.run_async_blocked(rod.K)
        with pytest.raises(H.Heat1dError) as ei:
            h.sync()
        assert ei.value.code == H.ERR_TIMEOUT
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, halo_steps=16) as h:
        h.set_u(rod.u0)
        h.run_async_blocked(rod.K)
        h.sync()


# ----------------------------------------------------------------------------- periodic ring (Section 5.3)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,S,q,T,K", [(1000, 4, 3, 16, 800), (4099, 7, 2, 33, 700), (300, 100, 3, 1, 500),
                                       (30, 2, 3, 12, 200)])
def test_blocked_periodic_free_and_replay(H, dtype, N, S, q, T, K):
    """Free blocked runs on the ring against the oracle through their traces,
    and seeded replays; (30, 2, T = 12) has a two-segment ring whose halos
    share points."""
    npdt = np.float32 if dtype == "float32" else np.float64
    rng = np.random.default_rng(N + S)
    u0 = rng.uniform(-1, 1, size=N)
    with H.Heat1d(N, 0.45, 0.0, 0.0, dtype=dtype, segments=S, q=q, halo_steps=T, boundary=1) as h:
        tr = h.new_blocked_trace(K)
        assert tuple(tr.shape) == (nblocks(K, T), S, 2)
        h.set_u(u0)
        h.run_async_blocked(K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
        assert trh.max() < q
        assert np.array_equal(got, oracle.async_blocked_periodic(u0, 0.45, S, q, T, K, trh, dtype=npdt))
        seeded = inputs.periodic_delay_trace(nblocks(K, T), S, q, seed=9)
        h.set_u(u0)
        h.replay_blocked(K, seeded)
        h.sync()
        assert np.array_equal(h.get_u(device=False),
                              oracle.async_blocked_periodic(u0, 0.45, S, q, T, K, seeded, dtype=npdt))
        h.set_u(u0)
        h.replay_blocked(K, np.zeros((nblocks(K, T), S, 2), dtype=np.uint8))
        h.sync()
        assert np.array_equal(h.get_u(device=False), oracle.sync_periodic(u0, 0.45, K, dtype=npdt))

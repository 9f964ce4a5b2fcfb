"""GPU parity of the asynchronous run with temporal blocking streamed through
HBM (the tiles of the streamed run are the segments of the blocked model).

Every free run is replayed by the oracle's blocked model on the tile split
the library reports (heat1d_blocked_segments), with the delay trace the GPU
recorded, and must agree bit for bit (FP64, and FP32 against the oracle's
float mode).  Replays of the recorded trace and of seeded traces reproduce
the oracle; an all-zero trace gives the synchronous run.  Small rods cover
tile shapes, block lengths that do not divide K, a last tile shorter than the
block length and single-tile rods; the 2^26-point rod is checked in full at
K = 200.  A tile that never publishes makes its neighbours' waits run out
(HEAT1D_ERR_TIMEOUT), and a trace entry >= q is rejected (HEAT1D_ERR_TRACE).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs
from tests import oracle_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch  # noqa: F401
    from paper_1510_08982_gb300 import build, heat1d
    build.build()
    return heat1d


def np_dt(dtype):
    return np.float32 if dtype == "float32" else np.float64


def free_run(H, rod, K, dtype, q=3, **opts):
    opts.setdefault("sync_mode", 2)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, q=q, **opts) as h:
        off, T = h.blocked_segments()
        h.set_u(rod.u0)
        tr = h.new_blocked_trace(K)
        h.run_async_blocked(K, tr)
        h.sync()
        return h.get_u(device=False), tr.cpu().numpy(), off, T


def replay(H, rod, K, trace, dtype, q=3, **opts):
    opts.setdefault("sync_mode", 2)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, q=q, **opts) as h:
        h.set_u(rod.u0)
        h.replay_blocked(K, np.ascontiguousarray(trace, dtype=np.uint8))
        h.sync()
        return h.get_u(device=False)


def oracle_replay(rod, off, q, T, K, trace, dtype):
    return oracle.async_blocked_split(rod.u0, rod.r, rod.c1, rod.cN, off, q, T, K, trace, dtype=np_dt(dtype))


def check(got, ref):
    assert got.dtype == ref.dtype
    err = float(np.abs(got.astype(np.float64) - ref.astype(np.float64)).max())
    assert np.array_equal(got, ref), "not bit-identical (max err %g)" % err


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,K,T,E,threads,q", [
    (5000, 300, 8, 8, 64, 3), (5003, 301, 17, 8, 64, 2), (20000, 500, 1, 8, 128, 3),
    (77777, 123, 64, 16, 256, 4), (3000, 40, 4, 4, 64, 1), (600, 90, 8, 8, 64, 3),
])
def test_streamed_async_free_run_replayed_by_oracle(H, dtype, N, K, T, E, threads, q):
    if dtype == "float64" and E == 16 and threads > 512:
        pytest.skip("shape not available in FP64")
    rng = np.random.default_rng(N + K + T)
    rod = inputs.Rod(N=N, K=K, r=0.41, c1=0.3, cN=-0.7, u0=rng.uniform(-1, 1, size=N))
    got, tr, off, Tb = free_run(H, rod, K, dtype, q=q, halo_steps=T, elems_per_thread=E, block_threads=threads)
    assert Tb == T and off[0] == 0 and off[-1] == N and tr.max(initial=0) < q
    check(got, oracle_replay(rod, off, q, T, K, tr, dtype))
    # the replay of the recorded trace is the same run
    check(replay(H, rod, K, tr, dtype, q=q, halo_steps=T, elems_per_thread=E, block_threads=threads), got)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_streamed_async_seeded_trace_and_short_last_tile(H, dtype):
    """A seeded trace (delays i.i.d. in {0..q-1}), a last tile of 3 points and
    a block length that does not divide K."""
    T, E, threads, q = 16, 8, 64, 3
    with H.Heat1d(100_000, 0.25, 0, 0, dtype=dtype, sync_mode=2, halo_steps=T, elems_per_thread=E,
                  block_threads=threads) as h0:
        W = int(h0.blocked_segments()[0][1])  # the tile width of this shape
    N = 7 * W + 3
    rng = np.random.default_rng(5)
    rod = inputs.Rod(N=N, K=203, r=0.33, c1=-0.2, cN=0.9, u0=rng.uniform(-1, 1, size=N))
    with H.Heat1d(N, rod.r, rod.c1, rod.cN, dtype=dtype, sync_mode=2, halo_steps=T, elems_per_thread=E,
                  block_threads=threads, q=q) as h:
        off, Tb = h.blocked_segments()
    assert off[-1] - off[-2] == 3 and Tb == T
    nb = (rod.K + T - 1) // T
    tr = inputs.delay_trace(nb, off.size - 1, q, seed=9)
    got = replay(H, rod, rod.K, tr, dtype, q=q, halo_steps=T, elems_per_thread=E, block_threads=threads)
    check(got, oracle_replay(rod, off, q, T, rod.K, tr, dtype))
    # all strips current: the synchronous run
    zero = np.zeros_like(tr)
    got0 = replay(H, rod, rod.K, zero, dtype, q=q, halo_steps=T, elems_per_thread=E, block_threads=threads)
    check(got0, oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K, dtype=np_dt(dtype)))


@pytest.mark.parametrize("dtype,T,K", [("float32", 1, 200), ("float32", 4, 300), ("float64", 2, 200),
                                       ("float32", 8, 160)])
def test_streamed_async_default_tiles_in_place_last_tile(H, dtype, T, K):
    """The default tile shape on a 2^22-point rod, block lengths at or below
    the warp-halo refresh depth (the compute warps then meet no barrier), a
    last tile of 128 to 3600 points read and written in place: free run and
    replay of its trace, both against the oracle."""
    rod = inputs.uniform_rod(N=1 << 22, K=K, seed=4)
    u0 = rod.u0.astype(np_dt(dtype)).astype(np.float64)
    rod = inputs.Rod(N=rod.N, K=K, r=rod.r, c1=0.0, cN=0.0, u0=u0)
    got, tr, off, Tb = free_run(H, rod, K, dtype, halo_steps=T)
    assert off[-1] - off[-2] >= 100  # a last tile of some length, read and written in place
    ref = oracle_replay(rod, off, 3, T, K, tr, dtype)
    check(got, ref)
    check(replay(H, rod, K, tr, dtype, halo_steps=T), ref)


def test_streamed_async_single_tile(H):
    rng = np.random.default_rng(3)
    rod = inputs.Rod(N=300, K=77, r=0.5, c1=1.0, cN=0.0, u0=rng.uniform(0, 1, size=300))
    got, tr, off, T = free_run(H, rod, rod.K, "float64", halo_steps=8, elems_per_thread=8, block_threads=64)
    assert off.size == 2 and tr.size == 0
    check(got, oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K))


@pytest.mark.parametrize("dtype,T", [("float32", 64), ("float64", 32), ("float32", 1)])
def test_streamed_async_full_size_rod(H, dtype, T):
    """Bandwidth / temporal-blocking rod: N = 2^26, c1 = cN = 0, u(0) ~ U[0,1),
    K = 200, free run replayed by the oracle bit for bit."""
    import torch
    rod = inputs.uniform_rod(K=200, seed=1)
    q = 3
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, sync_mode=2, halo_steps=T, q=q) as h:
        off, Tb = h.blocked_segments()
        u0 = torch.tensor(rod.u0.astype(np_dt(dtype)), device="cuda")
        h.set_u(u0)
        tr = h.new_blocked_trace(rod.K)
        h.run_async_blocked(rod.K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
    assert Tb == T and off.size - 1 > 1000
    hist = np.bincount(trh.reshape(-1), minlength=q)
    u0h = rod.u0.astype(np_dt(dtype)).astype(np.float64) if dtype == "float32" else rod.u0
    ref = oracle_pool.run([("async_blocked_split", (u0h, rod.r, rod.c1, rod.cN, off, q, T, rod.K, trh),
                            {"dtype": np_dt(dtype)})])[0]
    print("streamed async %s T=%d: %d tiles, delay histogram %s" % (dtype, T, off.size - 1, hist.tolist()))
    check(got, ref)


def test_streamed_async_stalled_tile_times_out(H):
    rod = inputs.uniform_rod(N=200_000, K=400, seed=2)
    with H.Heat1d(rod.N, rod.r, 0.0, 0.0, dtype="float32", sync_mode=2, halo_steps=16, stall_segment=5,
                  spin_limit_ns=200_000_000) as h:
        h.set_u(rod.u0.astype(np.float32))
        h.run_async_blocked(rod.K)
        with pytest.raises(H.Heat1dError) as ei:
            h.sync()
        assert ei.value.code == H.ERR_TIMEOUT
        # the handle stays usable
        h.set_opts(sync_mode=2, halo_steps=16)
        h.set_u(rod.u0.astype(np.float32))
        h.run_sync(rod.K)
        h.sync()


def test_streamed_async_bad_trace_is_rejected(H):
    rod = inputs.uniform_rod(N=50_000, K=64, seed=3)
    with H.Heat1d(rod.N, rod.r, 0.0, 0.0, dtype="float64", sync_mode=2, halo_steps=8, q=2) as h:
        h.set_u(rod.u0)
        tr = np.zeros(h.blocked_trace_bytes(rod.K), dtype=np.uint8)
        tr[len(tr) // 2] = 2
        h.replay_blocked(rod.K, tr)
        with pytest.raises(H.Heat1dError) as ei:
            h.sync()
        assert ei.value.code == H.ERR_TRACE

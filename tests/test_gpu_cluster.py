"""GPU parity of the per-step asynchronous run with thread-block clusters.

Neighbouring segments in one cluster hand their edge values to each other
through distributed shared memory; segments in different clusters through
the global rings.  Either way the run is Section 3's Eq. (eqn:async): every
free run, whatever the cluster size, must be reproduced bit for bit by the
oracle's replay of the delays it recorded, and a replay must give the same
state with clusters and without.  Cluster sizes 1, 2, 4 and 8 are forced on
rods where all segments share one cluster, where clusters meet (mixed
exchange paths), on the periodic ring (the wrap inside one cluster, or
between clusters), in FP32 and FP64, for resumed runs and for a stalled
segment inside a cluster.  The blocked run (strips of T points once per
block, the same clusters) is checked the same way against the oracle's
blocked model.
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


def np_dt(dtype):
    return np.float32 if dtype == "float32" else np.float64


def rod_of(N, K, seed):
    rng = np.random.default_rng(seed)
    return inputs.Rod(N=N, K=K, r=0.43, c1=-0.4, cN=0.8, u0=rng.uniform(-1, 1, size=N))


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,S,C,q,K", [
    (1024, 8, 8, 3, 3000),   # the small rod's shape: one cluster holds every segment
    (1024, 8, 1, 3, 3000),   # the same without clusters
    (5000, 16, 4, 3, 700),   # four clusters: both exchange paths
    (5001, 16, 8, 2, 700),
    (999, 6, 2, 3, 500),
    (4096, 32, 8, 4, 400),
    (20000, 4, 2, 1, 200),   # q = 1: no delay at all
])
def test_cluster_free_run_replayed_by_oracle(H, dtype, N, S, C, q, K):
    rod = rod_of(N, K, N + S + C)
    with H.Heat1d(N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q, cluster=C) as h:
        assert h.async_cluster() == C
        h.set_u(rod.u0)
        tr = h.new_trace(K)
        h.run_async(K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
        assert trh.max(initial=0) < q
        ref = oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, q, K, trh, dtype=np_dt(dtype))
        assert np.array_equal(got, ref)
        # the replay of the recorded delays, with this cluster size and without clusters
        h.set_u(rod.u0)
        h.replay(K, trh)
        h.sync()
        assert np.array_equal(h.get_u(device=False), got)
    with H.Heat1d(N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q, cluster=1) as h1:
        assert h1.async_cluster() == 1
        h1.set_u(rod.u0)
        h1.replay(K, trh)
        h1.sync()
        assert np.array_equal(h1.get_u(device=False), got)


@pytest.mark.parametrize("C", [8, 4, 1])
def test_cluster_seeded_replay_small_rod(H, C):
    """The small rod (N = 1024, r = 0.4, S = 8, q = 3, delays i.i.d. in
    {0,1,2} from seed 0) replayed through each exchange path."""
    rod = inputs.small_rod()
    tr = inputs.delay_trace(rod.K, 8, 3, seed=0)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, cluster=C) as h:
        h.set_u(rod.u0)
        h.replay(rod.K, tr)
        h.sync()
        got = h.get_u(device=False)
    assert np.array_equal(got, oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, rod.K, tr))


@pytest.mark.parametrize("N,S,C,q,K", [(1000, 8, 8, 3, 900), (1000, 8, 4, 3, 900), (64, 2, 2, 5, 500),
                                       (4000, 16, 4, 2, 300)])
def test_cluster_periodic_free_and_replay(H, N, S, C, q, K):
    """The ring of Section 5.3: with C = S the wrap-around boundary is inside
    the cluster, otherwise it joins the last cluster to the first."""
    rng = np.random.default_rng(N * S + C)
    u0 = rng.uniform(-1, 1, size=N)
    with H.Heat1d(N, 0.5, 0.0, 0.0, segments=S, q=q, boundary=1, cluster=C) as h:
        assert h.async_cluster() == C
        h.set_u(u0)
        tr = h.new_trace(K)
        h.run_async(K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
        assert np.array_equal(got, oracle.async_periodic(u0, 0.5, S, q, K, trh))
        seeded = inputs.periodic_delay_trace(K, S, q, seed=5)
        h.set_u(u0)
        h.replay(K, seeded)
        h.sync()
        assert np.array_equal(h.get_u(device=False), oracle.async_periodic(u0, 0.5, S, q, K, seeded))


@pytest.mark.parametrize("C", [8, 2])
def test_cluster_resumed_replay_equals_one_call(H, C):
    """A replay split into three calls (the later ones resume from the edge
    history the earlier ones left) equals the uninterrupted oracle replay."""
    rod = rod_of(2048, 600, 11)
    S, q = 8, 3
    tr = inputs.delay_trace(rod.K, S, q, seed=4)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=S, q=q, cluster=C) as h:
        h.set_u(rod.u0)
        for a, b in ((0, 1), (1, 250), (250, rod.K)):
            h.replay(b - a, np.ascontiguousarray(tr[a:b]))
        h.sync()
        got = h.get_u(device=False)
    assert np.array_equal(got, oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, q, rod.K, tr))


def test_cluster_stalled_segment_times_out(H):
    """A segment inside a cluster that never hands its edges on: its cluster
    neighbours' waits run out and the run ends with HEAT1D_ERR_TIMEOUT; the
    handle stays usable."""
    rod = inputs.small_rod(K=1000)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, cluster=8, stall_segment=3,
                  spin_limit_ns=200_000_000) as h:
        h.set_u(rod.u0)
        h.run_async(rod.K)
        with pytest.raises(H.Heat1dError) as ei:
            h.sync()
        assert ei.value.code == H.ERR_TIMEOUT
        h.set_opts(segments=8, q=3, cluster=8)
        h.set_u(rod.u0)
        h.run_sync(rod.K)
        h.sync()
        assert np.array_equal(h.get_u(device=False), oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K))


# --------------------------------------------------------------------------- blocked run


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,S,C,q,T,K", [
    (1024, 8, 8, 3, 32, 3000),   # the small rod's shape, one cluster
    (1024, 8, 1, 3, 32, 3000),
    (5000, 16, 4, 3, 16, 1000),  # clusters meet: strips through both paths
    (4099, 8, 2, 2, 33, 777),    # a block length that divides neither K nor the segments
    (2000, 4, 4, 5, 100, 1234),
])
def test_cluster_blocked_free_run_replayed_by_oracle(H, dtype, N, S, C, q, T, K):
    rod = rod_of(N, K, 3 * N + S + C)
    with H.Heat1d(N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q, halo_steps=T, cluster=C) as h:
        assert h.async_cluster(blocked=True) == C
        tr = h.new_blocked_trace(K)
        h.set_u(rod.u0)
        h.run_async_blocked(K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
        assert trh.max(initial=0) < q
        ref = oracle.async_blocked(rod.u0, rod.r, rod.c1, rod.cN, S, q, T, K, trh, dtype=np_dt(dtype))
        assert np.array_equal(got, ref)
        h.set_u(rod.u0)
        h.replay_blocked(K, tr)
        h.sync()
        assert np.array_equal(h.get_u(device=False), got)
    with H.Heat1d(N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q, halo_steps=T, cluster=1) as h1:
        h1.set_u(rod.u0)
        h1.replay_blocked(K, np.ascontiguousarray(trh))
        h1.sync()
        assert np.array_equal(h1.get_u(device=False), got)


@pytest.mark.parametrize("S,C", [(8, 8), (8, 2)])
def test_cluster_blocked_periodic_seeded_replay(H, S, C):
    N, q, T, K = 1200, 3, 20, 900
    rng = np.random.default_rng(S + C)
    u0 = rng.uniform(-1, 1, size=N)
    nb = (K + T - 1) // T
    tr = inputs.periodic_delay_trace(nb, S, q, seed=7)
    with H.Heat1d(N, 0.5, 0.0, 0.0, segments=S, q=q, halo_steps=T, boundary=1, cluster=C) as h:
        assert h.async_cluster(blocked=True) == C
        h.set_u(u0)
        h.replay_blocked(K, tr)
        h.sync()
        got = h.get_u(device=False)
    assert np.array_equal(got, oracle.async_blocked_periodic(u0, 0.5, S, q, T, K, tr))


def test_cluster_blocked_stalled_segment_times_out(H):
    rod = inputs.small_rod(K=2000)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3, halo_steps=16, cluster=8, stall_segment=5,
                  spin_limit_ns=200_000_000) as h:
        h.set_u(rod.u0)
        h.run_async_blocked(rod.K)
        with pytest.raises(H.Heat1dError) as ei:
            h.sync()
        assert ei.value.code == H.ERR_TIMEOUT


def test_cluster_option_checks(H):
    with pytest.raises(H.Heat1dError) as ei:
        H.Heat1d(1000, 0.3, 0.0, 0.0, segments=6, cluster=4)  # does not divide S
    assert ei.value.code == H.ERR_INVAL
    with pytest.raises(H.Heat1dError) as ei:
        H.Heat1d(1000, 0.3, 0.0, 0.0, segments=8, cluster=3)
    assert ei.value.code == H.ERR_INVAL
    with H.Heat1d(1000, 0.3, 0.0, 0.0, segments=7) as h:
        assert h.async_cluster() == 1  # 7 has no divisor among 8, 4, 2
    with H.Heat1d(1000, 0.3, 0.0, 0.0, segments=1, cluster=0) as h:
        assert h.async_cluster() == 1

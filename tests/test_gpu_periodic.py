"""GPU parity of the periodic boundary (Section 5.3): the synchronous ring
and the asynchronous ring (S boundaries) against the oracle, bit for bit."""
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


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,S,T,K", [(1000, 1, 64, 777), (1000, 3, 5, 777), (4099, 8, 1, 300), (100, 100, 1, 500),
                                     (64, 2, 32, 1000)])
def test_periodic_sync_bitwise(H, dtype, N, S, T, K):
    rng = np.random.default_rng(N + S)
    u0 = rng.uniform(-1, 1, size=N)
    with H.Heat1d(N, 0.37, 0.0, 0.0, dtype=dtype, segments=S, halo_steps=T, boundary=1) as h:
        h.set_u(u0)
        h.run_sync(K)
        h.sync()
        got = h.get_u(device=False)
    ref = oracle.sync_periodic(u0, 0.37, K, dtype=np.float32 if dtype == "float32" else np.float64)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("N,S,q,K", [(1000, 4, 3, 800), (100, 100, 3, 2000), (5000, 7, 2, 300), (64, 2, 5, 500)])
def test_periodic_async_free_and_replay(H, N, S, q, K):
    rng = np.random.default_rng(N * S)
    u0 = rng.uniform(-1, 1, size=N)
    with H.Heat1d(N, 0.5, 0.0, 0.0, segments=S, q=q, boundary=1) as h:
        h.set_u(u0)
        tr = h.new_trace(K)
        assert tuple(tr.shape) == (K, S, 2)
        h.run_async(K, tr)
        h.sync()
        got = h.get_u(device=False)
        trh = tr.cpu().numpy()
        assert trh.max() < q
        assert np.array_equal(got, oracle.async_periodic(u0, 0.5, S, q, K, trh))
        seeded = inputs.periodic_delay_trace(K, S, q, seed=3)
        h.set_u(u0)
        h.replay(K, seeded)
        h.sync()
        assert np.array_equal(h.get_u(device=False), oracle.async_periodic(u0, 0.5, S, q, K, seeded))


def test_periodic_paper_run_sum_drift(H):
    """The paper's periodic experiment (N = 100, one point per PE, r = 0.5,
    cos^2 start): the synchronous ring conserves the sum, the asynchronous
    ring does not (Fig. 6: no unique steady state)."""
    rod = inputs.paper_rod(N=100)
    K = 20000
    with H.Heat1d(100, 0.5, 0.0, 0.0, segments=100, q=3, boundary=1) as h:
        h.set_u(rod.u0)
        h.run_sync(K)
        h.sync()
        us = h.get_u(device=False)
        h.set_u(rod.u0)
        tr = h.new_trace(K)
        h.run_async(K, tr)
        h.sync()
        ua = h.get_u(device=False)
        trh = tr.cpu().numpy()
    assert abs(us.mean() - rod.u0.mean()) < 1e-13
    assert np.array_equal(ua, oracle.async_periodic(rod.u0, 0.5, 100, 3, K, trh))
    if trh.any():
        assert abs(ua.mean() - rod.u0.mean()) > 1e-12


def test_periodic_rejections(H):
    with H.Heat1d(1000, 0.25, 0.0, 0.0, segments=1, boundary=1) as h:
        with pytest.raises(H.Heat1dError):
            h.run_async(10)
    with pytest.raises(H.Heat1dError):
        H.Heat1d(1000, 0.25, 0.0, 0.0, boundary=1, sync_mode=2)

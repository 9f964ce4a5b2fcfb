"""GPU parity of the streamed synchronous run (temporal blocking through HBM)
against the CPU oracle.

Small rods: element by element, bit for bit, over tile shapes, halo depths,
step counts that are not multiples of the halo depth, and ragged tails.
Full-size rod (N = 2^26, K = 1e4): sampled outputs computed one by one by the
oracle on the cone that determines them.  u_i(K) depends only on u_{i-K..i+K}(0);
running the oracle on the window [i-K-1, i+K+1] with its two ends held fixed
gives u_i(K) exactly, because an error at a window end needs K+1 steps to
reach i.  Where the window meets a real Dirichlet end, that end is used.
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


def streamed(H, rod, K, dtype, **opts):
    opts.setdefault("sync_mode", 2)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, **opts) as h:
        h.set_u(rod.u0)
        h.run_sync(K)
        h.sync()
        return h.get_u(device=False)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("N,K,T,E,threads", [
    (3, 5, 1, 8, 32), (5, 7, 2, 8, 32), (1000, 100, 1, 8, 64), (1000, 101, 8, 8, 64),
    (4097, 333, 17, 8, 128), (100003, 250, 64, 16, 256), (65536, 64, 64, 4, 256), (77777, 123, 5, 16, 64),
])
def test_streamed_bitwise(H, dtype, N, K, T, E, threads):
    if dtype == "float64" and E == 16 and threads > 512:
        pytest.skip("shape not available in FP64")
    rng = np.random.default_rng(N + K)
    rod = inputs.Rod(N=N, K=K, r=0.37, c1=0.25, cN=-0.5, u0=rng.uniform(-1, 1, size=N))
    got = streamed(H, rod, K, dtype, halo_steps=T, elems_per_thread=E, block_threads=threads)
    ref = oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, K, dtype=np.float32 if dtype == "float32" else np.float64)
    assert np.array_equal(got, ref), float(np.abs(got.astype(np.float64) - ref).max())


def test_streamed_equals_on_chip(H):
    rod = inputs.sine_mode_rod(N=200_000, K=3000, seed=2, m_max=200)
    a = streamed(H, rod, rod.K, "float64", halo_steps=16)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype="float64", sync_mode=1) as h:
        h.set_u(rod.u0)
        h.run_sync(rod.K)
        h.sync()
        b = h.get_u(device=False)
    assert np.array_equal(a, b)


def cone_sample(u0, r, c1, cN, K, i, dtype):
    """u_i(K) from the oracle on the window that determines it."""
    N = u0.size
    lo, hi = max(0, i - K - 1), min(N - 1, i + K + 1)
    w = np.array(u0[lo:hi + 1], dtype=np.float64)
    # the real Dirichlet ends where the window reaches them; else the window
    # ends are held at their initial values (they cannot reach i in K steps)
    wc1 = c1 if lo == 0 else w[0]
    wcN = cN if hi == N - 1 else w[-1]
    out = oracle.sync(w, r, wc1, wcN, K, dtype=dtype)
    return out[i - lo]


@pytest.mark.parametrize("dtype,r,T", [("float32", 0.25, 16), ("float64", 0.5, 8)])
def test_streamed_full_size_sampled(H, dtype, r, T):
    """Bandwidth / temporal-blocking rod: N = 2^26, c1 = cN = 0, u(0) ~ U[0,1),
    K = 1e4, sampled outputs bit for bit (FP32 against the oracle's float
    mode), plus the maximum principle everywhere."""
    import torch
    rod = inputs.uniform_rod(r=r, seed=0)
    np_dt = np.float32 if dtype == "float32" else np.float64
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, sync_mode=2, halo_steps=T) as h:
        h.set_u(torch.tensor(rod.u0, dtype=torch.float32 if dtype == "float32" else torch.float64, device="cuda"))
        h.run_sync(rod.K)
        h.sync()
        got_t = h.get_u(device=True)
        assert float(got_t.min()) >= 0.0 and float(got_t.max()) <= 1.0
        samples = [0, 1, 5000, 1 << 25, (1 << 25) + 3999, rod.N - 9001, rod.N - 2, rod.N - 1]
        got = got_t[torch.tensor(samples, device="cuda")].cpu().numpy()
    u0 = rod.u0.astype(np_dt).astype(np.float64) if dtype == "float32" else rod.u0
    for i, g in zip(samples, got):
        ref = cone_sample(u0, rod.r, rod.c1, rod.cN, rod.K, i, np_dt)
        assert g == ref, (i, float(g), float(ref))


def test_streamed_stalled_tile_times_out(H):
    """A tile that never publishes its pass counter (a flag set on the host)
    makes its neighbours' bounded waits run out: the run ends with
    HEAT1D_ERR_TIMEOUT and the handle stays usable."""
    rod = inputs.uniform_rod(N=200_000, K=400, seed=2)
    with H.Heat1d(rod.N, rod.r, 0.0, 0.0, dtype="float32", sync_mode=2, halo_steps=16, stall_segment=5,
                  spin_limit_ns=200_000_000) as h:
        h.set_u(rod.u0.astype(np.float32))
        h.run_sync(rod.K)
        with pytest.raises(H.Heat1dError) as ei:
            h.sync()
        assert ei.value.code == H.ERR_TIMEOUT
        h.set_opts(sync_mode=2, halo_steps=16)
        h.set_u(rod.u0.astype(np.float32))
        h.run_sync(rod.K)
        h.sync()
        got = h.get_u(device=False)
    u0 = rod.u0.astype(np.float32)
    for i in (7, 123_456, rod.N - 2):
        assert got[i] == cone_sample(u0.astype(np.float64), rod.r, 0.0, 0.0, rod.K, i, np.float32)

"""Randomised GPU parity: seeded random shapes (rod length, segments, delay
window, halo depth, step count, precision, ends) through every on-chip run
of the library -- synchronous, asynchronous replay, blocked replay, and on
the periodic ring synchronous, asynchronous and blocked replay -- against
the oracle, bit for bit.

The shapes include the degenerate ones (N = 3, one point per segment, K = 0,
q = 1, T = 1, one segment) so that the corner cases of the segment split,
the warp windows and the delay bookkeeping are met on every run of the
suite.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = 40
EXTRA = 2  # N = 3: one segment, and three one-point segments


@pytest.fixture(scope="module")
def H():
    import torch  # noqa: F401
    from paper_1510_08982_gb300 import build, heat1d
    build.build()
    return heat1d


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    if seed >= CASES:  # the smallest rod: a single interior point
        S = 1 if seed == CASES else 3
        return 3, S, 3, 57, 1, "float64", 0.31, 0.5, -0.25, rng.uniform(-1, 1, size=3)
    kind = seed % 4
    if kind == 0:
        N = int(rng.integers(3, 40))
    elif kind == 1:
        N = int(rng.integers(40, 700))
    else:
        N = int(rng.integers(700, 6000))
    S = int(rng.integers(1, min(N, 160) + 1))
    if seed % 7 == 3:
        S = N if N <= 160 else S  # one point per segment
    q = int(rng.integers(1, 9))
    K = int(rng.integers(0, 400)) if seed % 5 else 0 if seed % 10 == 0 else int(rng.integers(1, 5))
    Lmin = N // S
    T = int(rng.integers(1, max(1, min(Lmin, 96)) + 1))
    dtype = "float32" if seed % 3 == 0 else "float64"
    r = float(rng.uniform(0.05, 0.5))
    c1, cN = (float(x) for x in rng.uniform(-1, 1, size=2))
    u0 = rng.uniform(-1, 1, size=N)
    return N, S, q, K, T, dtype, r, c1, cN, u0


@pytest.mark.parametrize("seed", range(CASES + EXTRA))
def test_random_shape_parity(H, seed):
    N, S, q, K, T, dtype, r, c1, cN, u0 = draw(seed)
    npdt = np.float32 if dtype == "float32" else np.float64
    rs, c1s, cNs = (float(np.float32(x)) if dtype == "float32" else x for x in (r, c1, cN))
    ctx = "N=%d S=%d q=%d K=%d T=%d %s" % (N, S, q, K, T, dtype)
    with H.Heat1d(N, r, c1, cN, dtype=dtype, segments=S, q=q, halo_steps=T, sync_mode=1) as h:
        h.set_u(u0)
        h.run_sync(K)
        h.sync()
        assert np.array_equal(h.get_u(device=False), oracle.sync(u0, rs, c1s, cNs, K, dtype=npdt)), ctx

        tr = inputs.delay_trace(K, S, q, seed=seed)
        h.set_u(u0)
        h.replay(K, tr)
        h.sync()
        ref = oracle.async_replay(u0, rs, c1s, cNs, S, q, K, tr if S > 1 else None, dtype=npdt)
        assert np.array_equal(h.get_u(device=False), ref), "replay " + ctx

        nb = (K + T - 1) // T
        btr = inputs.delay_trace(nb, S, q, seed=seed + 7)
        h.set_u(u0)
        h.replay_blocked(K, btr)
        h.sync()
        ref = oracle.async_blocked(u0, rs, c1s, cNs, S, q, T, K, btr if S > 1 else None, dtype=npdt)
        assert np.array_equal(h.get_u(device=False), ref), "blocked " + ctx

    if S >= 2:
        with H.Heat1d(N, r, 0.0, 0.0, dtype=dtype, segments=S, q=q, halo_steps=T, sync_mode=1, boundary=1) as h:
            h.set_u(u0)
            h.run_sync(K)
            h.sync()
            assert np.array_equal(h.get_u(device=False), oracle.sync_periodic(u0, rs, K, dtype=npdt)), \
                "periodic " + ctx
            ptr = inputs.periodic_delay_trace(K, S, q, seed=seed + 3)
            h.set_u(u0)
            h.replay(K, ptr)
            h.sync()
            ref = oracle.async_periodic(u0, rs, S, q, K, ptr, dtype=npdt)
            assert np.array_equal(h.get_u(device=False), ref), "periodic replay " + ctx
            pbtr = inputs.periodic_delay_trace((K + T - 1) // T, S, q, seed=seed + 5)
            h.set_u(u0)
            h.replay_blocked(K, pbtr)
            h.sync()
            ref = oracle.async_blocked_periodic(u0, rs, S, q, T, K, pbtr, dtype=npdt)
            assert np.array_equal(h.get_u(device=False), ref), "periodic blocked " + ctx

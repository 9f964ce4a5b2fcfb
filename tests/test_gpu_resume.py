"""Checkpoint and resume of the asynchronous run (heat1d_get_state /
heat1d_set_state): the augmented state of Section 3's Eq. (eqn:async) is u
plus every segment's edge values at the last q steps.  A run split into
several calls, through states copied to the host or kept on the device and
loaded into fresh handles, must equal the run made by one call bit for bit,
and both the oracle's replay of the concatenated trace."""
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


def make_rod(N, seed):
    rng = np.random.default_rng(seed)
    return inputs.Rod(N=N, K=0, r=0.42, c1=0.3, cN=-0.6, u0=rng.uniform(-1, 1, size=N))


@pytest.mark.parametrize("dtype,S,q,splits", [("float64", 8, 3, [0, 1, 57, 200]), ("float64", 16, 4, [0, 2, 3, 150]),
                                              ("float32", 7, 2, [0, 90, 91, 300]), ("float64", 5, 1, [0, 40, 120])])
def test_replay_split_into_calls_equals_one_call(H, dtype, S, q, splits):
    rod = make_rod(3001, S + q)
    K = splits[-1]
    tr = inputs.delay_trace(K, S, q, seed=7)
    np_dt = np.float32 if dtype == "float32" else np.float64
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q) as h:
        h.set_u(rod.u0)
        h.replay(K, tr)
        h.sync()
        whole = h.get_u(device=False)
    ref = oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, q, K, tr, dtype=np_dt)
    assert np.array_equal(whole, ref)
    # the same run in pieces, each piece in a fresh handle loaded from the previous state
    state = None
    for a, b in zip(splits[:-1], splits[1:]):
        with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q) as h:
            if state is None:
                h.set_u(rod.u0)
            else:
                h.set_state(state)
            if b > a:
                h.replay(b - a, np.ascontiguousarray(tr[a:b]))
            h.sync()
            state = h.get_state(device=(a % 2 == 1))
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, segments=S, q=q) as h:
        h.set_state(state)
        got = h.get_u(device=False)
    assert np.array_equal(got, whole)


def test_free_run_continued_is_one_run_of_eqn_async(H):
    """Free runs chained through a state: the concatenated recorded traces,
    replayed by the oracle, give the final state."""
    rod = make_rod(6000, 1)
    S, q = 12, 3
    traces = []
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=S, q=q) as h:
        h.set_u(rod.u0)
        for K in (1, 2, 333, 500):
            tr = h.new_trace(K)
            h.run_async(K, tr)
            h.sync()
            traces.append(tr.cpu().numpy())
            state = h.get_state()
            h.set_state(state)  # a round trip through the host changes nothing
        got = h.get_u(device=False)
    tr = np.concatenate(traces)
    assert tr.max() < q
    ref = oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, q, tr.shape[0], tr)
    assert np.array_equal(got, ref)


def test_periodic_replay_resumed(H):
    rng = np.random.default_rng(2)
    N, S, q, K = 1200, 6, 3, 240
    u0 = rng.uniform(0, 1, size=N)
    tr = inputs.periodic_delay_trace(K, S, q, seed=3)
    ref = oracle.async_periodic(u0, 0.35, S, q, K, tr)
    with H.Heat1d(N, 0.35, 0.0, 0.0, segments=S, q=q, boundary=1) as h:
        h.set_u(u0)
        h.replay(100, np.ascontiguousarray(tr[:100]))
        h.sync()
        st = h.get_state(device=True)
    with H.Heat1d(N, 0.35, 0.0, 0.0, segments=S, q=q, boundary=1) as h:
        h.set_state(st)
        h.replay(K - 100, np.ascontiguousarray(tr[100:]))
        h.sync()
        assert np.array_equal(h.get_u(device=False), ref)


def test_state_without_history_and_mismatched_handles(H):
    rod = make_rod(2000, 4)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3) as h:
        h.set_u(rod.u0)
        h.run_sync(10)            # no asynchronous history: the state starts a run
        st = h.get_state()
        u10 = h.get_u(device=False)
    hd = np.frombuffer(st[:48].tobytes(), dtype=np.int64)
    assert hd[1] == 0  # step
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3) as h:
        h.set_state(st)
        assert np.array_equal(h.get_u(device=False), u10)
        tr = inputs.delay_trace(50, 8, 3, seed=1)
        h.replay(50, tr)
        h.sync()
        assert np.array_equal(h.get_u(device=False), oracle.async_replay(u10, rod.r, rod.c1, rod.cN, 8, 3, 50, tr))
    for kw in (dict(segments=9, q=3), dict(segments=8, q=4)):
        with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, **kw) as h:
            with pytest.raises(H.Heat1dError) as ei:
                h.set_state(st)
            assert ei.value.code == H.ERR_INVAL
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype="float32", segments=8, q=3) as h:
        with pytest.raises(H.Heat1dError):
            h.set_state(st)

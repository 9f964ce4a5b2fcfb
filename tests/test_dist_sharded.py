"""One rod sharded over several gloo ranks on CPU: the host logic of the
multi-GPU path (chunks, neighbours, block schedule, strip history) with real
inter-process exchanges, checked bit for bit against the oracle.

Each rank owns chunk(N, W, rank) and, once per block of T steps, sends its
first and last T points to its neighbours and receives theirs; it then
advances its chunk with the T-wide halos (a tile whose outermost points are
held, the overlapped-halo trapezoid).  The stepping of a tile is the
oracle's synchronous run on that tile (its ends held = the tile edges), so
that the sharded run must equal the oracle's whole-rod run exactly:
  * every strip current  -> oracle.sync of the whole rod;
  * strips taken with the delays of a seeded trace (blocked asynchronous
    model, one segment per rank) -> oracle.async_blocked with S = W.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _exchange(rank, left, right, first, last, T):
    """Sends first/last T points to left/right and returns (from_left, from_right)."""
    reqs = []
    from_left = torch.zeros(T, dtype=torch.float64) if left >= 0 else None
    from_right = torch.zeros(T, dtype=torch.float64) if right >= 0 else None
    if left >= 0:
        reqs.append(dist.isend(torch.from_numpy(first.copy()), dst=left, tag=1))
        reqs.append(dist.irecv(from_left, src=left, tag=2))
    if right >= 0:
        reqs.append(dist.isend(torch.from_numpy(last.copy()), dst=right, tag=2))
        reqs.append(dist.irecv(from_right, src=right, tag=1))
    for rq in reqs:
        rq.wait()
    return (None if from_left is None else from_left.numpy().copy(),
            None if from_right is None else from_right.numpy().copy())


def _worker(rank, world, port, cfg, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1510_08982_gb300 import dist as hd
    N, K, T, q, r, c1, cN, seed, delayed = cfg
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-1, 1, size=N)
    u0[0], u0[-1] = c1, cN
    lo, hi = hd.chunk(N, world, rank)
    left, right = hd.neighbours(rank, world)
    u = u0[lo:hi].copy()
    nb = len(hd.blocks(K, T))
    from paper_1510_08982_gb300 import inputs
    trace = inputs.delay_trace(nb, world, q, seed=seed) if delayed else None
    hist_l, hist_r = hd.StripHistory(q), hd.StripHistory(q)
    for b, (k0, tb) in enumerate(hd.blocks(K, T)):
        fl, fr = _exchange(rank, left, right, u[:T], u[-T:], T)  # strips of version b
        if fl is not None:
            hist_l.put(b, fl)
        if fr is not None:
            hist_r.put(b, fr)
        dl = int(trace[b, rank - 1, 1]) if (delayed and left >= 0) else 0
        dr = int(trace[b, rank, 0]) if (delayed and right >= 0) else 0
        hl = hist_l.get(b, dl) if left >= 0 else np.zeros(0)
        hr = hist_r.get(b, dr) if right >= 0 else np.zeros(0)
        tile = np.concatenate([hl, u, hr])
        # tb steps with the tile's outermost points held; the rod's own ends are
        # the tile's ends on the first and last rank
        stepped = oracle.sync(tile, r, tile[0], tile[-1], tb)
        u = stepped[len(hl):len(hl) + (hi - lo)]
    parts = [torch.zeros(hd.chunk(N, world, k)[1] - hd.chunk(N, world, k)[0], dtype=torch.float64)
             for k in range(world)]
    if rank == 0:
        parts[0] = torch.from_numpy(u)
        for k in range(1, world):
            dist.recv(parts[k], src=k, tag=9)
        out.put(np.concatenate([p.numpy() for p in parts]))
    else:
        dist.send(torch.from_numpy(u), dst=0, tag=9)
    dist.barrier()
    dist.destroy_process_group()


def _run(world, cfg):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cfg, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = q.get(timeout=180)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world,N,K,T", [(2, 301, 57, 8), (3, 1000, 100, 16)])
def test_sharded_sync_equals_whole_rod(world, N, K, T):
    import oracle
    cfg = (N, K, T, 3, 0.37, 0.25, -0.5, 11, False)
    got = _run(world, cfg)
    rng = np.random.default_rng(11)
    u0 = rng.uniform(-1, 1, size=N)
    assert np.array_equal(got, oracle.sync(u0, 0.37, 0.25, -0.5, K))


def test_sharded_blocked_async_equals_oracle():
    import oracle
    from paper_1510_08982_gb300 import dist as hd
    from paper_1510_08982_gb300 import inputs
    world, N, K, T, q = 3, 400, 90, 7, 3
    cfg = (N, K, T, q, 0.41, 0.1, 0.9, 5, True)
    got = _run(world, cfg)
    rng = np.random.default_rng(5)
    u0 = rng.uniform(-1, 1, size=N)
    trace = inputs.delay_trace(len(hd.blocks(K, T)), world, q, seed=5)
    assert trace.any()
    assert np.array_equal(got, oracle.async_blocked(u0, 0.41, 0.1, 0.9, world, q, T, K, trace))


def test_sharded_per_step_async_equals_eqn_async():
    """Blocks of one step over two gloo ranks (one point-wide strips, delays per
    step): the run of Eq. (eqn:async) with one segment per rank, bit for bit."""
    import oracle
    from paper_1510_08982_gb300 import inputs
    world, N, K, q = 2, 120, 40, 3
    cfg = (N, K, 1, q, 0.45, -0.3, 0.6, 8, True)
    got = _run(world, cfg)
    rng = np.random.default_rng(8)
    u0 = rng.uniform(-1, 1, size=N)
    trace = inputs.delay_trace(K, world, q, seed=8)
    assert trace.any()
    assert np.array_equal(got, oracle.async_replay(u0, 0.45, -0.3, 0.6, world, q, K, trace))


def test_strip_history_and_plan():
    from paper_1510_08982_gb300 import dist as hd
    assert [hd.chunk(10, 3, k) for k in range(3)] == [(0, 4), (4, 7), (7, 10)]
    assert hd.neighbours(0, 3) == (-1, 1) and hd.neighbours(2, 3) == (1, -1)
    assert hd.neighbours(0, 3, periodic=True) == (2, 1)
    assert hd.blocks(10, 4) == [(0, 4), (4, 4), (8, 2)]
    h = hd.StripHistory(3)
    for v in range(6):
        h.put(v, v)                      # holds versions 3, 4, 5
    assert h.get(5, 0) == 5 and h.get(5, 2) == 3
    with pytest.raises(KeyError):
        h.get(2, 0)                      # dropped: older than the window
    with pytest.raises(ValueError):
        h.get(5, 3)                      # delay outside the window
    h0 = hd.StripHistory(3)
    h0.put(0, "v0")
    assert h0.get(1, 2) == "v0"          # clamped: no version before 0

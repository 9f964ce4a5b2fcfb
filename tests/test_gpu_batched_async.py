"""GPU parity of the asynchronous batched run.

The parts of every rod that is split over several CTAs are the segments of
the blocked asynchronous model (Eq. (eqn:async) per block of T steps, strips
up to q-1 blocks old; the oracle's split model, since parts are uneven).  A
free run is replayed by the oracle rod by rod from the delays the GPU
recorded and must agree bit for bit; so must a replay of the recorded trace
and of seeded traces; an all-zero trace gives the synchronous batch; rods
that are not split come out as the synchronous oracle.  Small CTAs force many
parts on short rods.  A part that never publishes makes its neighbours time
out; a delay >= q is rejected.
"""
from __future__ import annotations

import math

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


def make_rods(n, seed, N_lo=200, N_hi=3000, K_lo=50, K_hi=700):
    rng = np.random.default_rng(seed)
    rods = []
    for _ in range(n):
        N = int(rng.integers(N_lo, N_hi))
        K = int(rng.integers(K_lo, K_hi))
        rods.append(inputs.Rod(N=N, K=K, r=float(rng.uniform(0.05, 0.5)), c1=float(rng.uniform(-1, 1)),
                               cN=float(rng.uniform(-1, 1)), u0=rng.uniform(-1, 1, size=N)))
    return rods


def pack(H, rods, dtype):
    import torch
    off, total = H.pack_offsets([r.N for r in rods])
    u = np.zeros(total)
    for o, r in zip(off, rods):
        u[o:o + r.N] = r.u0
    specs = [(int(o), r.N, r.K, r.r, r.c1, r.cN) for o, r in zip(off, rods)]
    tdt = torch.float64 if dtype == "float64" else torch.float32
    return specs, torch.tensor(u.astype(np_dt(dtype)), dtype=tdt, device="cuda"), off


def rod_trace(b, j, rod, T, trace):
    """The oracle's trace of rod j ([ceil(K/T)][P-1][2]: side 0 part b's read
    of its right neighbour, side 1 part b+1's read of its left neighbour)
    from the batch's part-by-part trace, with the part offsets."""
    offs, toff = b.rod_parts(j)
    P = offs.size - 1
    if P == 1:
        return offs, None
    nb = math.ceil(rod.K / T)
    parts = trace[toff:toff + 2 * P * nb].reshape(P, nb, 2)
    tr = np.zeros((nb, P - 1, 2), dtype=np.uint8)
    for bnd in range(P - 1):
        tr[:, bnd, 0] = parts[bnd, :, 1]
        tr[:, bnd, 1] = parts[bnd + 1, :, 0]
    return offs, tr


def oracle_rod(rod, offs, tr, q, T, dtype):
    u0 = rod.u0.astype(np_dt(dtype)).astype(np.float64) if dtype == "float32" else rod.u0
    if tr is None:
        return oracle.sync(u0, rod.r, rod.c1, rod.cN, rod.K, dtype=np_dt(dtype))
    return oracle.async_blocked_split(u0, rod.r, rod.c1, rod.cN, offs, q, T, rod.K, tr, dtype=np_dt(dtype))


SHAPES = {"float64": dict(elems_per_thread=4, block_threads=128), "float32": dict(elems_per_thread=4, block_threads=128)}


@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("q,T", [(3, 16), (2, 5), (4, 32)])
def test_batched_async_free_run_replayed_by_oracle(H, dtype, q, T):
    rods = make_rods(24, seed=q * 100 + T)
    specs, u, off = pack(H, rods, dtype)
    with H.Batch(specs, dtype=dtype, q=q, halo_steps=T, **SHAPES[dtype]) as b:
        info = b.describe()
        assert info["rod_parts"] > 20
        tr = b.new_trace()
        b.run_async(u, tr)
        b.sync()
        got = u.cpu().numpy()
        trh = tr.cpu().numpy()
        assert trh.max(initial=0) < q
        split = 0
        for j, (o, r) in enumerate(zip(off, rods)):
            offs, rtr = rod_trace(b, j, r, T, trh)
            split += rtr is not None
            if rtr is not None:
                assert not rtr[0].any()  # block 0 reads only version 0
            ref = oracle_rod(r, offs, rtr, q, T, dtype)
            assert np.array_equal(got[o:o + r.N], ref), (j, r.N, r.K, offs.size - 1)
        assert split >= 10
        # the replay of the recorded trace is the same run
        _, u2, _ = pack(H, rods, dtype)
        b.replay(u2, tr)
        b.sync()
        assert np.array_equal(u2.cpu().numpy(), got)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_batched_async_seeded_and_zero_traces(H, dtype):
    import torch
    q, T = 3, 8
    rods = make_rods(16, seed=7)
    specs, u, off = pack(H, rods, dtype)
    with H.Batch(specs, dtype=dtype, q=q, halo_steps=T, **SHAPES[dtype]) as b:
        n = b.trace_bytes()
        seeded = np.random.default_rng(11).integers(0, q, size=n).astype(np.uint8)
        b.replay(u, torch.tensor(seeded, device="cuda"))
        b.sync()
        got = u.cpu().numpy()
        for j, (o, r) in enumerate(zip(off, rods)):
            offs, rtr = rod_trace(b, j, r, T, seeded)
            if rtr is not None:
                rtr = rtr.copy()
                rtr[0] = 0  # block 0 reads version 0 whatever the entry says
            assert np.array_equal(got[o:o + r.N], oracle_rod(r, offs, rtr, q, T, dtype)), j
        # all delays zero: the synchronous batch
        _, u0, _ = pack(H, rods, dtype)
        b.replay(u0, torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda"))
        b.sync()
        _, us, _ = pack(H, rods, dtype)
        b.run(us)
        b.sync()
        assert np.array_equal(u0.cpu().numpy(), us.cpu().numpy())


def test_batched_async_in_a_cuda_graph(H):
    import torch
    q, T = 3, 16
    rods = make_rods(12, seed=3)
    specs, u, off = pack(H, rods, "float64")
    with H.Batch(specs, dtype="float64", q=q, halo_steps=T, **SHAPES["float64"]) as b:
        tr = b.new_trace()
        seeded = torch.tensor(np.random.default_rng(2).integers(0, q, size=tr.numel()).astype(np.uint8),
                              device="cuda")
        u_start = u.clone()
        b.replay(u, seeded)  # first asynchronous run: allocates the strip rings outside the capture
        b.sync()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                b.replay(u, seeded)
        for _ in range(2):
            u.copy_(u_start)
            g.replay()
        torch.cuda.synchronize()
        b.sync()
        got = u.cpu().numpy()
        sh = seeded.cpu().numpy()
        for j, (o, r) in enumerate(zip(off, rods)):
            offs, rtr = rod_trace(b, j, r, T, sh)
            if rtr is not None:
                rtr = rtr.copy()
                rtr[0] = 0
            assert np.array_equal(got[o:o + r.N], oracle_rod(r, offs, rtr, q, T, "float64")), j


def test_batched_async_failures(H):
    import torch
    rods = make_rods(6, seed=5, N_lo=2000)
    specs, u, off = pack(H, rods, "float64")
    # a part that never publishes: its neighbours time out
    with H.Batch(specs, dtype="float64", q=3, halo_steps=16, stall_segment=1, spin_limit_ns=200_000_000,
                 **SHAPES["float64"]) as b:
        b.run_async(u)
        with pytest.raises(H.Heat1dError) as ei:
            b.sync()
        assert ei.value.code == H.ERR_TIMEOUT
    # a delay >= q in a replay
    specs, u, off = pack(H, rods, "float64")
    with H.Batch(specs, dtype="float64", q=2, halo_steps=16, **SHAPES["float64"]) as b:
        bad = np.full(b.trace_bytes(), 2, dtype=np.uint8)  # every read of a neighbour out of the window
        b.replay(u, torch.tensor(bad, device="cuda"))
        with pytest.raises(H.Heat1dError) as ei:
            b.sync()
        assert ei.value.code == H.ERR_TRACE

"""GPU parity of the batched persistent launch (many uneven rods at once).

Every rod of a batch must come out bit-identical to the oracle run on that rod
alone.  Small batches cover all three kinds of work item (warp batches,
single-CTA rods, multi-CTA parts) and degenerate rods; the uneven-rods
workload (4096 rods, N log-uniform in [256, 65536], K log-uniform in
[1e3, 1e5]) is checked against the oracle on a seeded subset and on its six
heaviest rods.
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


def pack(H, rods, dtype):
    import torch
    off, total = H.pack_offsets([r.N for r in rods])
    u = np.zeros(total)
    for o, r in zip(off, rods):
        u[o:o + r.N] = r.u0
    tdt = torch.float64 if dtype == "float64" else torch.float32
    specs = [(int(o), r.N, r.K, r.r, r.c1, r.cN) for o, r in zip(off, rods)]
    return specs, torch.tensor(u, dtype=tdt, device="cuda"), off


def oracle_rod(r, dtype):
    return oracle.sync(r.u0, r.r, r.c1, r.cN, r.K, dtype=np.float32 if dtype == "float32" else np.float64)


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_batched_all_item_kinds(H, dtype):
    rng = np.random.default_rng(11)
    Ns = [3, 4, 17, 100, 127, 128, 129, 200, 251, 300, 777, 1000, 2500, 6000, 3, 50]
    Ks = [5, 0, 7, 100, 1000, 1, 33, 250, 64, 999, 17, 8, 300, 77, 1, 2000]
    rods = [inputs.Rod(N=N, K=K, r=float(rng.uniform(0.05, 0.5)), c1=float(rng.uniform(-1, 1)),
                       cN=float(rng.uniform(-1, 1)), u0=rng.uniform(-1, 1, size=N)) for N, K in zip(Ns, Ks)]
    specs, u, off = pack(H, rods, dtype)
    with H.Batch(specs, dtype=dtype, elems_per_thread=4, block_threads=64, halo_steps=8) as b:
        info = b.describe()
        assert info["warp_batches"] > 0 and info["cta_rods"] > 0 and info["rod_parts"] > 0, info
        b.run(u)
        b.sync()
    got = u.cpu().numpy()
    for o, r in zip(off, rods):
        g = got[o:o + r.N]
        if r.K == 0:
            assert np.array_equal(g, r.u0.astype(g.dtype))
            continue
        ref = oracle_rod(r, dtype)
        assert np.array_equal(g, ref), (r.N, r.K, float(np.abs(g.astype(np.float64) - ref).max()))


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_batched_uneven_rods_workload(H, dtype):
    """4096 uneven rods in one launch: a seeded subset of 64 cheap rods and
    the 6 heaviest rods against the oracle."""
    rods = inputs.uneven_rods(seed=0)
    specs, u, off = pack(H, rods, dtype)
    with H.Batch(specs, dtype=dtype) as b:
        info = b.describe()
        b.run(u)
        b.sync()
    assert info["rod_parts"] > 0 and info["warp_batches"] > 0
    got = u.cpu().numpy()
    cheap = [j for j, r in enumerate(rods) if r.N * r.K <= 2e7]
    pick = np.random.default_rng(1).choice(cheap, size=64, replace=False)
    for j in pick:
        r = rods[j]
        assert np.array_equal(got[off[j]:off[j] + r.N], oracle_rod(r, dtype)), j
    # the six heaviest rods (N up to 65536, K up to 1e5, split into parts
    # over several CTAs) against the oracle, in parallel worker processes
    big = sorted(range(len(rods)), key=lambda j: rods[j].N * rods[j].K)[-6:]
    odt = np.float32 if dtype == "float32" else np.float64
    refs = oracle_pool.run([("sync", (rods[j].u0, rods[j].r, rods[j].c1, rods[j].cN, rods[j].K), {"dtype": odt})
                            for j in big])
    for j, ref in zip(big, refs):
        r = rods[j]
        assert r.N > 8192 and r.K > 20_000
        assert np.array_equal(got[off[j]:off[j] + r.N], ref), j


def test_batched_in_a_cuda_graph(H):
    import torch
    rods = inputs.uneven_rods(n_rods=300, seed=5, K_hi=3000)
    specs, u0, off = pack(H, rods, "float32")
    with H.Batch(specs, dtype="float32") as b:
        ref = u0.clone()
        b.run(ref)
        b.sync()
        u = u0.clone()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                b.run(u)
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(2):
            u.copy_(u0)
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(u, ref)
        b.sync()


def test_batched_rejects_bad_rods(H):
    with pytest.raises(H.Heat1dError):
        H.Batch([(0, 100, 10, 0.75, 0.0, 0.0)], dtype="float64")
    with pytest.raises(H.Heat1dError):
        H.Batch([(0, 2, 10, 0.25, 0.0, 0.0)], dtype="float64")


def test_batched_stalled_part_times_out(H):
    """A rod part that never publishes its epochs (a flag set on the host)
    makes its neighbours' bounded waits run out: HEAT1D_ERR_TIMEOUT; a batch
    planned without the flag then runs correctly."""
    rng = np.random.default_rng(4)
    rods = [inputs.Rod(N=30_000, K=300, r=0.3, c1=0.1, cN=-0.2, u0=rng.uniform(-1, 1, size=30_000))
            for _ in range(3)]
    specs, u, off = pack(H, rods, "float64")
    with H.Batch(specs, dtype="float64", stall_segment=2, spin_limit_ns=200_000_000) as b:
        assert b.describe()["rod_parts"] > 3
        b.run(u)
        with pytest.raises(H.Heat1dError) as ei:
            b.sync()
        assert ei.value.code == H.ERR_TIMEOUT
    specs, u, off = pack(H, rods, "float64")
    with H.Batch(specs, dtype="float64") as b:
        b.run(u)
        b.sync()
    got = u.cpu().numpy()
    for o, r in zip(off, rods):
        assert np.array_equal(got[o:o + r.N], oracle_rod(r, "float64"))

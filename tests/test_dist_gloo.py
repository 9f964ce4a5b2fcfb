"""The multi-rank path on CPU: two gloo ranks run the bench's rank logic
(distinct rods per rank, sharded batches, max-over-ranks timing, whole-job
rate) with no GPU."""
from __future__ import annotations

import os
import socket

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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1510_08982_gb300 import dist as hd
    from paper_1510_08982_gb300 import inputs
    r, w, lr = hd.env()
    rod = inputs.sine_mode_rod(N=4096, K=10, seed=hd.rod_seed(r))
    lo, hi = hd.shard(4096, r, w)
    # pretend rank r took (r+1) seconds: the job time is the slowest rank's
    t = hd.max_over_ranks(float(r + 1), w)
    rate = hd.whole_job_rate((rod.N - 2) * rod.K, t, w)
    # gather what each rank saw
    mine = torch.tensor([float(rod.u0[1]), lo, hi, t, rate], dtype=torch.float64)
    allv = [torch.zeros_like(mine) for _ in range(w)]
    dist.all_gather(allv, mine)
    if r == 0:
        out.put([v.tolist() for v in allv])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_run_the_rank_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (u0a, lo0, hi0, t0, rate0), (u0b, lo1, hi1, t1, rate1) = res
    assert u0a != u0b                      # each rank runs its own rod
    assert (lo0, hi0, lo1, hi1) == (0, 2048, 2048, 4096)
    assert t0 == t1 == 2.0                 # max over ranks
    assert rate0 == rate1 == 2 * (4096 - 2) * 10 / 2.0


def test_shard_covers_everything_once():
    from paper_1510_08982_gb300 import dist as hd
    for n in (0, 1, 7, 4096, 4099):
        for w in (1, 2, 3, 8):
            parts = [hd.shard(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))

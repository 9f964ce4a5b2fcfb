"""Rank logic of multi-GPU runs (one process per GPU, launched by torchrun).

The path shards by independent rods: every rank advances its own rod(s) with
no collective on the data path (weak scaling).  The only communication is
host-side bookkeeping: barriers around the timed region and the maximum of
the ranks' times, from which the whole-job throughput is computed.
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rod_seed(rank: int, base: int = 1000) -> int:
    """Seed of the rank's synthetic rod: distinct per rank, fixed per run."""
    return base + rank


def shard(n_items: int, rank: int, world: int):
    """Contiguous share [lo, hi) of n_items for this rank (first n % world
    ranks get one more) -- used to split a batch of independent rods."""
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank value (the slowest rank's time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max: float, world: int) -> float:
    """Whole-job throughput: the units every rank processed divided by the
    slowest rank's time.  units_per_rank: a number (same on every rank) or a
    list with one entry per rank."""
    total = units_per_rank * world if isinstance(units_per_rank, (int, float)) else sum(units_per_rank)
    return total / seconds_max

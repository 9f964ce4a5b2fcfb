"""Rank logic of multi-GPU runs (one process per GPU, launched by torchrun).

The benchmark shards by independent rods: every rank advances its own rod(s)
with no collective on the data path (weak scaling).  The only communication
there is host-side bookkeeping: barriers around the timed region and the
maximum of the ranks' times, from which the whole-job throughput is computed.

One rod can also be sharded: rank k owns the contiguous chunk ``chunk(N, W,
k)`` (the paper's PE decomposition of Fig. 1 with one PE per GPU) and trades
T-wide edge strips with its two neighbours once per block of T steps
(``blocks``): synchronously (every strip current) or in the blocked
asynchronous model (a strip up to q-1 blocks old, ``StripHistory``).  These
helpers hold that protocol's host logic; the exchange itself is a send and a
receive per neighbour and block.
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


# ----------------------------------------------------------------------------- one rod over several ranks


def chunk(N: int, world: int, rank: int):
    """Contiguous points [lo, hi) of rank `rank` when one rod of N points is
    split over `world` ranks (the first N % world ranks get one more point,
    the rule of the segment split)."""
    return shard(N, rank, world)


def neighbours(rank: int, world: int, periodic: bool = False):
    """(left, right) neighbour ranks of a chunk; -1 where the rod ends."""
    left = rank - 1 if rank > 0 else (world - 1 if periodic and world > 1 else -1)
    right = rank + 1 if rank + 1 < world else (0 if periodic and world > 1 else -1)
    return left, right


def blocks(K: int, T: int):
    """The blocks of a run of K steps, T steps per exchange: (first step,
    steps) pairs, the last one possibly shorter."""
    if T < 1:
        raise ValueError("T must be >= 1")
    return [(k0, min(T, K - k0)) for k0 in range(0, K, T)]


class StripHistory:
    """The last q strips received from one neighbour, by version (version b =
    the neighbour's edge at the start of block b).  ``get(b, d)`` returns the
    strip that block b reads with delay d (clamped to b, as no strip is older
    than version 0) and fails loudly if it is not held."""

    def __init__(self, q: int):
        if q < 1:
            raise ValueError("q must be >= 1")
        self.q = q
        self._strips = {}

    def put(self, version: int, strip):
        self._strips[version] = strip
        for v in [v for v in self._strips if v <= version - self.q]:
            del self._strips[v]

    def get(self, block: int, delay: int):
        if delay >= self.q:
            raise ValueError("delay %d outside the window q = %d" % (delay, self.q))
        v = block - min(delay, block)
        if v not in self._strips:
            raise KeyError("strip version %d is not held" % v)
        return self._strips[v]

"""Runs oracle calls in parallel worker processes (test infrastructure).

The full-size parity tests replay GPU runs of 1e9 to 1e11 grid-point updates
through the single-threaded CPU oracle.  Independent oracle calls (the
synchronous sweep, the replay of a trace, the blocked replay, one rod of a
batch) run in separate processes at once.  Workers are started with the
"spawn" method: a process forked from one that already holds a CUDA context
can hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def _call(job):
    import oracle
    name, args, kwargs = job
    return getattr(oracle, name)(*args, **kwargs)


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def run(jobs, processes=None):
    """jobs: list of (oracle function name, args tuple, kwargs dict); returns
    the results in order."""
    n = max(1, min(len(jobs), processes or host_cores()))
    if n == 1:
        return [_call(j) for j in jobs]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_call, jobs, chunksize=1)


def start(jobs, processes=None):
    """Starts the jobs without waiting; returns (pool, AsyncResult).  The
    caller closes the pool after .get()."""
    n = max(1, min(len(jobs), processes or host_cores()))
    pool = mp.get_context("spawn").Pool(n)
    return pool, pool.map_async(_call, jobs, chunksize=1)


def available_host_bytes() -> int:
    """Host memory currently available (MemAvailable of /proc/meminfo)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")

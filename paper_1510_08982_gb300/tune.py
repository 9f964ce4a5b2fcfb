"""Autotuner for the batched and streamed synchronous runs.

Tile shape (threads per CTA, points per thread E) and temporal-block depth T
do not change results (every configuration is bit-identical to one step at a
time), so they are picked purely by measurement:

* ``tune_batched(specs, dtype)``: times each candidate (E, threads, T) on a
  sample of the batch stratified by rod size (the sample keeps the batch's mix
  of warp-batch rods, single-CTA rods and multi-CTA rods, with K capped so that
  tuning takes seconds) and returns the fastest as options for ``Batch``.
* ``tune_stream(N, dtype)``: times each candidate (E, threads, T) on the
  streamed run of an N-point rod for a few passes.

Results are cached in a JSON file (``HEAT1D_TUNE_CACHE``, default
``~/.cache/heat1d_tune.json``) keyed by GPU name, dtype and the workload's size
classes, so a batch with the same shape is tuned once.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from . import heat1d

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("HEAT1D_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "heat1d_tune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store_cache(key: str, value: dict) -> None:
    with _lock:
        c = _load_cache()
        c[key] = value
        p = cache_path()
        os.makedirs(os.path.dirname(p) or ".", exist_ok=True)
        tmp = p + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, p)


def size_classes(Ns, Ks) -> str:
    """Histogram of rods by log2(N) and log10(K) buckets, as a compact key."""
    nb = np.clip(np.floor(np.log2(np.maximum(Ns, 2))).astype(int), 0, 40)
    kb = np.clip(np.floor(np.log10(np.maximum(Ks, 1))).astype(int), 0, 12)
    h = {}
    for a, b in zip(nb, kb):
        h["%d.%d" % (a, b)] = h.get("%d.%d" % (a, b), 0) + 1
    total = len(Ns)
    # bucket shares rounded to 5 %, so that batches of the same shape share a key
    return ",".join("%s:%d" % (k, round(20 * v / total)) for k, v in sorted(h.items()) if round(20 * v / total))


def batched_candidates(dtype: str):
    if dtype in ("float64", "f64"):
        return [dict(elems_per_thread=e, block_threads=t, halo_steps=T)
                for e in (4, 8) for t in (128, 256) for T in (8, 16, 32)]
    return [dict(elems_per_thread=e, block_threads=t, halo_steps=T)
            for e in (8, 16) for t in (128, 256, 512) for T in (64, 128, 256)]


def stream_candidates(dtype: str):
    if dtype in ("float64", "f64"):
        return [dict(elems_per_thread=e, block_threads=t, halo_steps=T)
                for e in (4, 8) for t in (128, 256) for T in (8, 16, 32, 64)]
    return [dict(elems_per_thread=e, block_threads=t, halo_steps=T)
            for e in (8, 16) for t in (128, 256) for T in (16, 64, 128, 192)]


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _sample_specs(specs, n_sample: int, k_cap: int):
    """Stratified sample: rods sorted by N, evenly spaced picks, K capped."""
    order = sorted(range(len(specs)), key=lambda j: specs[j][1])
    if len(order) > n_sample:
        idx = np.linspace(0, len(order) - 1, n_sample).round().astype(int)
        order = [order[j] for j in idx]
    Ns = [int(specs[j][1]) for j in order]
    off, total = heat1d.pack_offsets(Ns)
    out = [(int(o), int(specs[j][1]), int(min(specs[j][2], k_cap)), float(specs[j][3]), float(specs[j][4]),
            float(specs[j][5])) for o, j in zip(off, order)]
    return out, total


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batched(specs, dtype="float32", n_sample=256, k_cap=2000, reps=2, use_cache=True, candidates=None):
    """Options (elems_per_thread, block_threads, halo_steps) for ``Batch``
    that ran fastest on a stratified sample of ``specs`` (offset, N, K, r,
    c1, cN)."""
    import torch
    Ns = np.array([s[1] for s in specs])
    Ks = np.array([s[2] for s in specs])
    key = "batched|%s|%s|%s" % (_gpu_name(), dtype, size_classes(Ns, Ks))
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit["opts"])
    sample, total = _sample_specs(specs, n_sample, k_cap)
    tdt = torch.float64 if dtype in ("float64", "f64") else torch.float32
    u0 = torch.rand(total, dtype=tdt, device="cuda")
    u = torch.empty_like(u0)
    updates = sum((s[1] - 2) * s[2] for s in sample)
    results = []
    for opts in (candidates or batched_candidates(dtype)):
        try:
            b = heat1d.Batch(sample, dtype="float64" if tdt == torch.float64 else "float32", **opts)
        except heat1d.Heat1dError:
            continue

        def run():
            u.copy_(u0)
            b.run(u)

        ms = _time(run, reps)
        b.sync()
        b.close()
        results.append((updates / (ms * 1e-3), opts))
    if not results:
        raise RuntimeError("no batched configuration could be planned")
    best = max(results, key=lambda x: x[0])
    if use_cache:
        _store_cache(key, {"opts": best[1], "updates_per_s": best[0],
                           "tried": [[float(v), o] for v, o in results]})
    return dict(best[1])


def tune_stream(N, dtype="float32", passes=4, reps=2, use_cache=True, candidates=None):
    """Options (elems_per_thread, block_threads, halo_steps) for the streamed
    synchronous run of an N-point rod that ran fastest over a few passes."""
    import torch
    key = "stream|%s|%s|%d" % (_gpu_name(), dtype, int(math.log2(max(N, 2))))
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit["opts"])
    tdt = torch.float64 if dtype in ("float64", "f64") else torch.float32
    u0 = torch.rand(N, dtype=tdt, device="cuda")
    results = []
    for opts in (candidates or stream_candidates(dtype)):
        try:
            h = heat1d.Heat1d(N, 0.25, 0.0, 0.0, dtype="float64" if tdt == torch.float64 else "float32",
                              sync_mode=2, **opts)
        except heat1d.Heat1dError:
            continue
        K = passes * opts["halo_steps"]

        def run():
            h.set_u(u0)
            h.run_sync(K)

        ms = _time(run, reps)
        h.sync()
        h.close()
        results.append(((N - 2) * K / (ms * 1e-3), opts))
    best = max(results, key=lambda x: x[0])
    if use_cache:
        _store_cache(key, {"opts": best[1], "updates_per_s": best[0],
                           "tried": [[float(v), o] for v, o in results]})
    return dict(best[1])

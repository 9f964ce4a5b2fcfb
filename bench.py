"""Benchmark: grid-point updates/s of the synchronous and asynchronous FTCS
runs on one GB300 per rank.

Workload (the "sync vs async at scale" rod): N = 2^20 points in FP64,
r = 0.25, c1 = -1, cN = 1, K = 1e5 steps, u(0) a sum of 16 sine modes
(m uniform in [1, 512], amplitudes N(0, 1), seed = 1000 + rank), one segment
per SM, delay window q = 3.

One bench step is one pass of the whole path on that rod:
  set-up (u(0) copied into the handle, ends forced)
  -> synchronous run of K steps (persistent kernel, grid barrier every T steps)
  -> asynchronous run of K steps (no barrier), delay trace recorded on device
  -> replay of that trace (exact re-execution) .
Updates per step = 3 * (N-2) * K.

Under torchrun each rank runs its own rod on its own GPU (independent problems,
no collective on the data path: weak scaling).  The CPU oracle arm
(``--impl reference``) times the plain C oracle on a bounded sample of the
same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s, async vs sync, at stated error; % of HBM/SMEM roofline"
UNIT = "updates/s"
N_DEFAULT = 1 << 20
K_DEFAULT = 100_000
Q = 3
# FP64 pipe: 1.25 TFLOP/s nominal for GB300 (recipe table) = 6.25e11 FP64
# instructions/s at 2070 MHz; one update issues 3 of them (3 DFMA: the middle
# add is issued as a fused multiply-add by one).
FP64_NOMINAL_TFLOPS = 1.25
FP64_INSTR_PER_UPDATE = 3
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of one launch of the asynchronous kernel on the
# 2^20-point rod, from the committed ncu summary of that kernel.
ASYNC_KERNEL_DRAM_BYTES = 8_503_552 + 1_792
# DRAM bytes (read + write) per pass of the streamed kernel on the 2^26-point
# FP32 rod, from the committed ncu summary (T = 1: 4 passes, T = 128: 2
# passes); a launch makes ceil(K/T) passes of the same traffic.
STREAM_F32_DRAM_BYTES_PER_PASS = {1: (1_077_127_000 + 1_026_632_000) / 4, 128: (539_179_008 + 487_579_136) / 2}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=N_DEFAULT)
    p.add_argument("--K", type=int, default=K_DEFAULT)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default="sine-mode-rod",
                   choices=["sine-mode-rod", "small-rod", "streamed-rod", "uneven-rods", "inverse-problem"],
                   help="sine-mode-rod (default): the sync vs async rod; streamed-rod: the 2^26-point "
                        "temporal-blocking rod; uneven-rods: 4096 rods in one batched launch")
    p.add_argument("--dtype", default=None, choices=["f32", "f64"], help="streamed-rod / uneven-rods precision")
    p.add_argument("--halo", type=int, default=0, help="streamed-rod: steps per HBM pass (T)")
    p.add_argument("--r", type=float, default=0.25, help="streamed-rod: r (the sweep's values are 0.1, 0.25, 0.5)")
    p.add_argument("--rods", type=int, default=256, help="inverse-problem: rods in the batch")
    p.add_argument("--async-trace", action="store_true", help="inverse-problem: replayed asynchronous run")
    return p.parse_args()


def dist_env():
    from paper_1510_08982_gb300 import dist as hd
    return hd.env()


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arm


def oracle_sample(rod, seconds=10.0, S=152, all_cores=False):
    """Times the plain C oracle (single thread) on a bounded sample of the
    workload: the synchronous sweep and the asynchronous replay on the full N
    for Ks steps, Ks chosen for about `seconds` of CPU work.  With `all_cores`
    the same sample, at half the steps, also runs as one process per host core
    (the host's aggregate rate)."""
    import oracle
    N = rod.N
    probe = 4
    tr = np.zeros((probe, S - 1, 2), dtype=np.uint8)
    t0 = time.perf_counter()
    oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, probe)
    oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, Q, probe, tr)
    per_step = (time.perf_counter() - t0) / probe
    Ks = max(2, int(seconds / max(per_step, 1e-9)))
    from paper_1510_08982_gb300 import inputs
    tr = inputs.delay_trace(Ks, S, Q, seed=0)
    t0 = time.perf_counter()
    oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, Ks)
    oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, Q, Ks, tr)
    dt = time.perf_counter() - t0
    updates = 2 * (N - 2) * Ks
    out = {"value": updates / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "plain C oracle, one thread: synchronous sweep + asynchronous replay (seeded q=3 delays, "
                     "S=%d) of the N=%d rod for %d steps each (%.1f s)" % (S, N, Ks, dt)}
    if all_cores:
        out["all_cores"] = oracle_all_cores(rod, S, max(2, Ks // 2))
    return out


_ORACLE_JOB = None


def _oracle_init(job):
    global _ORACLE_JOB
    import oracle  # noqa: F401  (loaded before the timed region)
    _ORACLE_JOB = job


def _oracle_job(_):
    import oracle
    u0, r, c1, cN, S, Ks, tr = _ORACLE_JOB
    oracle.sync(u0, r, c1, cN, Ks)
    oracle.async_replay(u0, r, c1, cN, S, Q, Ks, tr)
    return os.getpid()


def oracle_all_cores(rod, S, Ks):
    """The same single-threaded oracle sample run as one process per host core
    at once (spawned workers, inputs handed over before the clock starts):
    the aggregate updates/s of the host.  None on a one-core host."""
    import multiprocessing as mp
    P = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    if P < 2:
        return None
    from paper_1510_08982_gb300 import inputs
    job = (rod.u0, rod.r, rod.c1, rod.cN, S, Ks, inputs.delay_trace(Ks, S, Q, seed=0))
    with mp.get_context("spawn").Pool(P, initializer=_oracle_init, initargs=(job,)) as pool:
        t0 = time.perf_counter()
        pids = pool.map(_oracle_job, range(P), chunksize=1)
        dt = time.perf_counter() - t0
    updates = P * 2 * (rod.N - 2) * Ks
    return {"value": updates / dt, "cores": P, "processes_used": len(set(pids)),
            "sample": "%d concurrent copies of the one-thread sample, %d steps each (%.1f s wall)" % (P, Ks, dt)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1510_08982_gb300 import inputs
    rod = inputs.sine_mode_rod(N=args.N, K=args.K, seed=1000)
    for _ in range(args.warmup):
        oracle_sample(rod, seconds=1.0)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = oracle_sample(rod, seconds=8.0)
        vals.append(last["value"])
    wall = time.perf_counter() - t0
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, 152),
            "cpu_baseline": dict(last, value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm


def workload_config(args, S):
    return {"workload": "sine-mode rod: N=%d FP64, r=0.25, c1=-1, cN=1, K=%d, 16 modes m~U[1,512] A~N(0,1), "
                        "S=%d segments (one per SM), q=%d; step = sync + async (trace recorded) + replay"
                        % (args.N, args.K, S, Q),
            "N": args.N, "K": args.K, "segments": S, "q": Q,
            "l2": "flushed between timed steps (256 MB write); the rod itself stays on-chip for the whole run"}


def hd_seed(rank):
    from paper_1510_08982_gb300 import dist as hd
    return hd.rod_seed(rank)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def _build_once(rank, world):
    """Builds the library (if stale) on rank 0 only; the other ranks wait, so
    that concurrent ranks never write the same object files."""
    from paper_1510_08982_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank != 0:
        build.build()  # up to date by now: only checks


def _device_setup():
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build_once(rank, world)
    return torch, rank, world, local


def _max_over_ranks(torch, world, x, dev):
    from paper_1510_08982_gb300 import dist as hd
    return hd.max_over_ranks(x, world, dev)


def run_streamed(args):
    """The 2^26-point rod (c1 = cN = 0, u(0) ~ U[0,1), r = --r, 0.25 by
    default, K = 1e4) advanced by the streamed synchronous run, T steps per HBM
    pass."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    dev = torch.device("cuda", local)
    dt = args.dtype or "f32"
    esz = 4 if dt == "f32" else 8
    K = args.K if args.K != K_DEFAULT else 10_000
    N = args.N if args.N != N_DEFAULT else 1 << 26
    T = args.halo or (128 if dt == "f32" else 32)
    tdt = torch.float32 if dt == "f32" else torch.float64
    g = torch.Generator(device=dev).manual_seed(hd_seed(rank))
    u0 = torch.rand(N, dtype=tdt, device=dev, generator=g)
    h = heat1d.Heat1d(N, args.r, 0.0, 0.0, dtype="float32" if dt == "f32" else "float64", sync_mode=2, halo_steps=T)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        h.set_u(u0)
        h.run_sync(K)
    h.sync()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    total = 0.0
    for _ in range(args.steps):
        h.set_u(u0)  # 2*N*esz bytes > L2: the rod itself flushes L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.run_sync(K)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    clk = clocks.stop()
    h.sync()
    total = _max_over_ranks(torch, world, total, dev)
    ms = total / args.steps
    ups = world * (N - 2) * K / (ms * 1e-3)
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alg_bytes = 2.0 * esz * N * (K / T)  # each pass reads and writes the rod once
    achieved_gbs = alg_bytes / (ms * 1e-3) / 1e9
    # ALU roofline: FP32 128 FMA-pipe lanes/clk/SM, FP64 1.25 TFLOP/s nominal (2 per SM per clk); 3 ops per update
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_ups = (nsm * 128 * 2.07e9 if dt == "f32" else FP64_NOMINAL_TFLOPS * 1e12 / 2) / 3
    hbm_ups = hbm * 1e9 / (2.0 * esz / T)
    bound = "hbm" if hbm_ups < alu_ups else "alu"
    roof = ({"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm}
            if bound == "hbm" else
            {"bound": "alu", "achieved": ups / 1e9, "peak": alu_ups / 1e9, "unit": "Gupdates/s",
             "frac": ups / alu_ups})
    per_pass = STREAM_F32_DRAM_BYTES_PER_PASS.get(T) if dt == "f32" and N == 1 << 26 else None
    traffic = None if per_pass is None else per_pass * math.ceil(K / T)
    roof.update({"kernel": "stream_tma_kernel", "peak_source": src, "traffic": traffic,
                 "traffic_source": None if traffic is None else
                 "ncu dram__bytes_read+write of this kernel on this rod, per pass x passes (profiles/)",
                 "hbm_roofline_updates_per_s": hbm_ups, "alu_roofline_updates_per_s": alu_ups,
                 "algorithmic_bytes_per_update": 2.0 * esz / T, "achieved_algorithmic_GBs": achieved_gbs})
    line = {"metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt, "data": "synthetic",
            "config": {"workload": "streamed rod: N=%d %s, r=%g, c1=cN=0, u(0)~U[0,1), K=%d, T=%d steps per "
                                   "HBM pass" % (N, dt.upper(), args.r, K, T), "N": N, "K": K, "T": T, "r": args.r,
                       "l2": "inputs larger than L2 (%d MB state)" % (N * esz >> 20)},
            "roofline": roof, "clocks": clk, "gpu_launches": 2 * args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_small(args):
    """The small rod (N = 1024 FP64, r = 0.4, c1 = 0, cN = 1, u(0) = sin(pi x) +
    0.5 sin(7 pi x) + x, S = 8, q = 3): latency-bound.  Per-step device times
    of the persistent synchronous run, the free asynchronous run, its replay,
    the asynchronous run with temporal blocking (the default block length: 32
    steps on these 128-point segments), and a
    synchronous run relaunched once per step (the paper's structure without its
    host copies); then async vs sync at equal error: the steps and the time to
    ||u(k) - u_ss||_inf <= 1e-6."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    dev = torch.device("cuda", local)
    rod = inputs.small_rod()
    N, S = rod.N, 8
    K = args.K if args.K != K_DEFAULT else rod.K
    eps, every = 1e-6, 1024
    h = heat1d.Heat1d(N, rod.r, rod.c1, rod.cN, dtype="float64", segments=S, q=Q)
    u0 = torch.tensor(rod.u0, dtype=torch.float64, device=dev)
    uss = torch.tensor(rod.c1 + (rod.cN - rod.c1) * inputs.grid_x(N), dtype=torch.float64, device=dev)
    tr = h.new_trace(K)
    stream = torch.cuda.current_stream()
    lib, hp = h.lib, h.h

    def relaunch(n):
        for _ in range(n):  # one launch per step, stream set once
            rc = lib.heat1d_run_sync(hp, 1)
            if rc:
                raise heat1d.Heat1dError(rc, heat1d.last_error())

    def timed(fn):
        h.set_u(u0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    btr = h.new_blocked_trace(K)
    runs = {"sync": lambda: h.run_sync(K), "async": lambda: h.run_async(K, tr), "replay": lambda: h.replay(K, tr),
            "async_blocked": lambda: h.run_async_blocked(K, btr), "sync_relaunch_per_step": lambda: relaunch(K)}
    for _ in range(args.warmup):
        for f in runs.values():
            timed(f)
    h.sync()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    tot = {k: 0.0 for k in runs}
    for _ in range(args.steps):
        for k, f in runs.items():
            tot[k] += timed(f)
    h.sync()
    # async vs sync at equal error: first snapshot at or below eps, then a timed run of that many steps
    lam1 = 1.0 - 4.0 * rod.r * math.sin(math.pi / (2.0 * (N - 1))) ** 2
    k_est = int(math.log(eps) / math.log(lam1))
    kmax = (int(1.25 * k_est) // every + 1) * every
    snaps = torch.empty((kmax // every + 1, N), dtype=torch.float64, device=dev)
    eq = {"eps": eps, "norm": "max abs of u(k) - u_ss", "snapshot_every": every,
          "closed_form_sync_steps": k_est}
    for kind, fn in (("sync", h.run_sync), ("async", h.run_async), ("async_blocked", h.run_async_blocked)):
        h.set_snapshots(snaps, every=every)
        h.set_u(u0)
        fn(kmax)
        h.sync()
        err = (snaps - uss).abs().amax(dim=1).cpu().numpy()
        h.set_snapshots(None)
        hit = np.nonzero(err <= eps)[0]
        if hit.size == 0:
            eq[kind] = None
            continue
        k_eps = int(hit[0]) * every
        t = timed(lambda: fn(k_eps))
        h.sync()
        err_end = float((h.get_u() - uss).abs().max())
        eq[kind] = {"steps": k_eps, "seconds": t, "error_at_end": err_end}
    if eq.get("sync"):
        eq["sync_relaunch_per_step"] = {"steps": eq["sync"]["steps"],
                                        "seconds": eq["sync"]["steps"] * tot["sync_relaunch_per_step"] / (args.steps * K),
                                        "note": "per-step time of the timed relaunch run x the synchronous steps"}
    clk = clocks.stop()
    us = {k: 1e6 * v / (args.steps * K) for k, v in tot.items()}
    upd = (N - 2) * K
    ups = {k: upd * args.steps / v for k, v in tot.items()}
    t_step = tot["sync"] + tot["async"] + tot["replay"]
    value = world * 3 * upd * args.steps / _max_over_ranks(torch, world, t_step, dev)
    peak_upd = FP64_NOMINAL_TFLOPS * 1e12 / 2 / FP64_INSTR_PER_UPDATE
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "small rod: N=1024 FP64, r=0.4, c1=0, cN=1, u(0)=sin(pi x)+0.5 sin(7 pi x)+x, "
                                   "K=%d, S=8, q=3; step = sync + async (trace recorded) + replay" % K,
                       "N": N, "K": K, "segments": S, "q": Q,
                       "l2": "the 8 KB rod stays on-chip; latency-bound, L2 state does not matter"},
            "us_per_step": us, "updates_per_s": ups,
            "blocked_delay_histogram": np.bincount(btr.cpu().numpy().reshape(-1), minlength=Q).tolist(),
            "speedup": {"async_vs_relaunch_per_step": us["sync_relaunch_per_step"] / us["async"],
                        "async_blocked_vs_relaunch_per_step": us["sync_relaunch_per_step"] / us["async_blocked"],
                        "persistent_sync_vs_relaunch_per_step": us["sync_relaunch_per_step"] / us["sync"]},
            "equal_error": eq,
            "roofline": {"bound": "alu", "kernel": "async_persistent_kernel<double,8>",
                         "achieved": ups["async"] / 1e9, "peak": peak_upd / 1e9, "unit": "Gupdates/s",
                         "frac": ups["async"] / peak_upd, "traffic": None,
                         "note": "8 CTAs on a 1024-point rod: bound by exchange latency, the ALU fraction is "
                                 "reported but not meaningful"},
            "clocks": clk, "gpu_launches": args.steps * (4 + K)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        trn = tr.cpu().numpy()
        t0 = time.perf_counter()
        oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, K)
        oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, Q, K, trn)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 2 * upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "plain C oracle, one thread: full synchronous run and replay of the "
                                          "recorded trace, K=%d (%.2f s)" % (K, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_uneven(args):
    """4096 uneven rods in one batched persistent launch, replayed from a CUDA graph."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    dev = torch.device("cuda", local)
    dt = args.dtype or "f32"
    esz = 4 if dt == "f32" else 8
    tdt = torch.float32 if dt == "f32" else torch.float64
    rods = inputs.uneven_rods(seed=hd_seed(rank))
    off, total_n = heat1d.pack_offsets([r.N for r in rods])
    host = np.zeros(total_n)
    for o, r in zip(off, rods):
        host[o:o + r.N] = r.u0
    u0 = torch.tensor(host, dtype=tdt, device=dev)
    u = u0.clone()
    specs = [(int(o), r.N, r.K, r.r, r.c1, r.cN) for o, r in zip(off, rods)]
    from paper_1510_08982_gb300 import tune
    opts = tune.tune_batched(specs, "float32" if dt == "f32" else "float64")  # cached per GPU and batch shape
    b = heat1d.Batch(specs, dtype="float32" if dt == "f32" else "float64", **opts)
    info = b.describe()
    updates = sum((r.N - 2) * r.K for r in rods)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            b.run(u)
    torch.cuda.current_stream().wait_stream(s)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        u.copy_(u0)
        graph.replay()
    torch.cuda.synchronize()
    b.sync()
    clocks = ClockSampler(local)
    clocks.start()
    total = 0.0
    for _ in range(args.steps):
        u.copy_(u0)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    clk = clocks.stop()
    b.sync()
    total = _max_over_ranks(torch, world, total, dev)
    ms = total / args.steps
    ups = world * updates / (ms * 1e-3)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_ups = (nsm * 128 * 2.07e9 if dt == "f32" else FP64_NOMINAL_TFLOPS * 1e12 / 2) / 3
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(total_n, dtype=tdt).pin_memory()
        pinned.copy_(torch.tensor(host, dtype=tdt))
        out = torch.empty_like(pinned).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            u.copy_(pinned, non_blocking=True)
            b.run(u)
            out.copy_(u, non_blocking=True)
            torch.cuda.synchronize()
        dt_e2e = (time.perf_counter() - t0) / args.steps
        b.sync()
        e2e = {"value": world * updates / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": total_n * esz,
               "d2h_bytes_per_step": total_n * esz, "path": "pinned host -> device, heat1d_batch_run, device -> host"}
    line = {"metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt, "data": "synthetic",
            "config": {"workload": "uneven rods: 4096 rods, N log-U[256,65536], K log-U[1e3,1e5], r U[0.05,0.5], "
                                   "8 sine modes; one batched persistent launch replayed from a CUDA graph; tile "
                                   "and halo depth from the autotuner",
                       "rods": len(rods), "points": total_n, "updates": updates, "plan": info,
                       "l2": "flushed between timed steps (256 MB write)"},
            "roofline": {"bound": "alu", "kernel": "batched_kernel", "achieved": ups / 1e9, "peak": alu_ups / 1e9,
                         "unit": "Gupdates/s", "frac": ups / alu_ups, "traffic": None},
            "clocks": clk, "e2e": e2e, "gpu_launches": args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    return 0


def run_inverse(args):
    """Adjoint of the inverse problem: 256 rods of N = 65536, K = 2e4, smooth
    u(0), r_true ~ U[0.1, 0.45], u_obs = u(K) + N(0, 1e-4); one step = the
    forward pass with checkpoints every 128 steps + the backward pass
    (recompute + transposed stencil), giving dL/du(0) and dL/dr per rod."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    dev = torch.device("cuda", local)
    dt = args.dtype or "f64"
    tdt = torch.float32 if dt == "f32" else torch.float64
    K = args.K if args.K != K_DEFAULT else 20_000
    N = args.N if args.N != N_DEFAULT else 65536
    nr = args.rods
    rods = inputs.inverse_problem_rods(n_rods=nr, N=N, K=K, seed=hd_seed(rank))
    u0 = torch.tensor(np.stack([r.u0 for r in rods]), dtype=tdt, device=dev)
    r = np.array([x.r for x in rods])
    c1 = np.array([x.c1 for x in rods])
    cN = np.array([x.cN for x in rods])
    S, q = 16, 3  # 4096 points per segment: one CTA each for the observation runs
    trace = None
    if args.async_trace:
        trace = torch.tensor(np.stack([inputs.delay_trace(K, S, q, seed=j) for j in range(nr)]), device=dev)
    # observations: u(K) at r_true plus noise; the gradient is taken at 0.9 r_true
    uobs = torch.empty(nr, N, dtype=torch.float64, device=dev)
    for j, x in enumerate(rods):
        opts = {"segments": S, "q": q} if trace is not None else {}
        with heat1d.Heat1d(N, x.r, x.c1, x.cN, dtype="float32" if dt == "f32" else "float64", **opts) as h:
            h.set_u(u0[j])
            if trace is None:
                h.run_sync(K)
            else:
                h.replay(K, trace[j].contiguous())
            h.sync()
            uobs[j] = h.get_u().double()
    uobs += torch.tensor(np.stack([inputs.observation_noise(N, seed=7000 + j) for j in range(nr)]), device=dev)
    rg = 0.9 * r

    def step():
        return heat1d.adjoint_batched(u0, uobs, rg, c1, cN, K, trace=trace, segments=S if trace is not None else 0,
                                      q=q, ckpt_every=128)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = step()
    torch.cuda.synchronize()
    dt_s = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    dt_s = _max_over_ranks(torch, world, dt_s, dev)
    updates = nr * (N - 2) * K
    ups = world * updates / dt_s
    # FP64: FP64-pipe instructions per forward update over the three passes:
    # 3 (forward) + 3 (recompute) + 4 (backward: t, the r-gradient term and
    # the lambda update, 2 + 1 + 1, where nothing is pending); the peak in
    # forward-equivalent updates/s.
    # FP32: u and lambda in FP32, every pass one launch per step over all rods
    # streaming its arrays: forward and recompute read u(k) and write u(k+1)
    # (8 bytes per point and step each), the backward reads u(k) and
    # lambda(k+1) and writes lambda(k) (12 bytes): 28 bytes per forward update
    # at the measured HBM rate.
    fp64_rate = FP64_NOMINAL_TFLOPS * 1e12 / 2
    if dt == "f64":
        bound, alu = "alu", fp64_rate / (3 + 3 + 4)
        roof_note = ("three passes per forward update: forward and recompute 3 FP64 instructions per point, "
                     "backward 4; peak = nominal FP64 instruction rate / 10")
    else:
        hbm = float(measured_peaks()[0].get("hbm_gbs", 6800.0)) * 1e9
        bound, alu = "hbm", hbm / 28.0
        roof_note = ("FP32 passes bound by HBM: forward 8 + recompute 8 + backward 12 bytes per point and step; "
                     "peak = measured HBM / 28 B, in forward-equivalent updates/s")
    line = {"metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt, "data": "synthetic",
            "config": {"workload": "inverse problem: %d rods x N=%d, K=%d, checkpoints every 128 steps, %s; one step = "
                                   "forward with checkpoints + backward (recompute + adjoint); value counts forward "
                                   "updates (rods x (N-2) x K) per second of the whole gradient computation"
                                   % (nr, N, K, "replayed trace S=16 q=3" if trace is not None else "synchronous"),
                       "rods": nr, "N": N, "K": K, "ckpt_every": 128},
            "gradient": {"grad_r_first_rods": [float(x) for x in out[2][:4]], "loss_first_rods": [float(x) for x in out[3][:4]]},
            "roofline": {"bound": bound, "kernel": "adj_fwd_step / adj_bwd_step", "achieved": ups / 1e9,
                         "peak": alu / 1e9, "unit": "Gupdates/s (forward-equivalent)", "frac": ups / alu,
                         "note": roof_note},
            "clocks": clk, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "streamed-rod":
        return run_streamed(args)
    if args.workload == "small-rod":
        return run_small(args)
    if args.workload == "uneven-rods":
        return run_uneven(args)
    if args.workload == "inverse-problem":
        return run_inverse(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1510_08982_gb300 import heat1d, inputs
    _build_once(rank, world)
    dev = torch.device("cuda", local)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    from paper_1510_08982_gb300 import dist as hd
    rod = inputs.sine_mode_rod(N=args.N, K=args.K, seed=hd.rod_seed(rank))
    N, K = rod.N, rod.K
    M = N - 2
    h = heat1d.Heat1d(N, rod.r, rod.c1, rod.cN, dtype="float64", segments=nsm, q=Q)
    S = h.S
    u0 = torch.tensor(rod.u0, dtype=torch.float64, device=dev)
    trace = h.new_trace(K)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def step(evs=None):
        """One pass: set-up, sync, async (trace), replay.  evs: 4 events
        bracketing the three runs on the launching stream."""
        h.set_u(u0)
        if evs:
            evs[0].record(stream)
        h.run_sync(K)
        if evs:
            evs[1].record(stream)
        h.set_u(u0)
        h.run_async(K, trace)
        if evs:
            evs[2].record(stream)
        h.set_u(u0)
        h.replay(K, trace)
        if evs:
            evs[3].record(stream)

    for _ in range(args.warmup):
        step()
    h.sync()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    t_sync = t_async = t_replay = total = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        e_begin = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e_begin.record(stream)
        step(evs)
        e_end.record(stream)
        e_end.synchronize()
        total += e_begin.elapsed_time(e_end)
        t_sync += evs[0].elapsed_time(evs[1])
        t_async += evs[1].elapsed_time(evs[2])
        t_replay += evs[2].elapsed_time(evs[3])
    barrier()
    clk = clocks.stop()
    h.sync()
    total = hd.max_over_ranks(total, world, dev)
    ms_per_step = total / args.steps
    updates_per_step = 3 * M * K
    value = hd.whole_job_rate(updates_per_step, ms_per_step * 1e-3, world)
    per = {name: M * K / (t / args.steps * 1e-3) for name, t in
           (("sync", t_sync), ("async", t_async), ("replay", t_replay))}

    # --- the blocked asynchronous run on the same rod (its own timing, not part of the step) --
    btr = h.new_blocked_trace(K)
    h.set_u(u0)
    h.run_async_blocked(K, btr)
    h.sync()
    t_blocked = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        h.set_u(u0)
        eb0 = torch.cuda.Event(enable_timing=True)
        eb1 = torch.cuda.Event(enable_timing=True)
        eb0.record(stream)
        h.run_async_blocked(K, btr)
        eb1.record(stream)
        eb1.synchronize()
        t_blocked += eb0.elapsed_time(eb1)
    h.sync()
    t_blocked = hd.max_over_ranks(t_blocked, world, dev)
    per["async_blocked"] = M * K / (t_blocked / args.steps * 1e-3)
    blocked_hist = np.bincount(btr.cpu().numpy().reshape(-1), minlength=Q)[:Q].tolist()

    # --- error at the stated tolerance (untimed) -----------------------------------------
    from scipy.fft import dst, idst
    h.set_u(u0)
    h.run_sync(K)
    h.sync()
    u_sync = h.get_u(device=False)
    x = np.arange(N) / (N - 1)
    uss = rod.c1 + (rod.cN - rod.c1) * x
    f = (np.where(np.arange(N) == 0, rod.c1, np.where(np.arange(N) == N - 1, rod.cN, rod.u0)) - uss)[1:-1]
    lam = 1.0 - 4.0 * rod.r * np.sin(np.arange(1, N - 1) * np.pi / (2.0 * (N - 1))) ** 2
    exact = uss.copy()
    exact[1:-1] += idst(dst(f, type=1) * np.exp(K * np.log(np.abs(lam))) * np.sign(lam) ** (K % 2), type=1)
    err_sync = float(np.abs(u_sync - exact).max())
    h.set_u(u0)
    h.run_async(K, trace)
    h.sync()
    u_async = h.get_u(device=False)
    h.set_u(u0)
    h.replay(K, trace)
    h.sync()
    replay_exact = bool(np.array_equal(h.get_u(device=False), u_async))
    async_vs_sync = float(np.abs(u_async - u_sync).max())
    tr_host = trace.cpu().numpy()
    hist = np.bincount(tr_host.reshape(-1), minlength=Q).tolist()

    # --- e2e through the C ABI with host buffers ------------------------------------------
    e2e = None
    if not args.no_e2e:
        u_host = torch.tensor(rod.u0, dtype=torch.float64).pin_memory().numpy()
        out_host = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        tr_h = torch.empty(trace.numel(), dtype=torch.uint8).pin_memory().numpy().reshape(trace.shape)

        def e2e_step():
            h.set_u(u_host)
            h.run_sync(K)
            h.get_u(out_host, device=False)
            h.set_u(u_host)
            h.run_async(K, tr_h)
            h.sync()
            h.get_u(out_host, device=False)
            h.set_u(u_host)
            h.replay(K, tr_h)
            h.sync()
            h.get_u(out_host, device=False)

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        dt = (time.perf_counter() - t0) / args.steps
        dt = hd.max_over_ranks(dt, world, dev)
        tb = trace.numel()
        e2e = {"value": world * updates_per_step / dt, "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * N + tb, "d2h_bytes_per_step": 3 * 8 * N + tb,
               "path": "heat1d_set_u/run_*/replay/get_u from pinned host buffers, host traces"}

    # --- roofline of the dominant kernel (the asynchronous persistent kernel) -------------
    peak_upd = FP64_NOMINAL_TFLOPS * 1e12 / 2 / FP64_INSTR_PER_UPDATE
    achieved = per["async"]
    roofline = {"bound": "alu", "kernel": "async_persistent_kernel<double,8>",
                "achieved": achieved / 1e9, "peak": peak_upd / 1e9, "unit": "Gupdates/s",
                "frac": achieved / peak_upd,
                "peak_source": "recipe nominal FP64 1.25 TFLOP/s at 2070 MHz = 6.25e11 FP64-pipe instr/s, "
                               "3 per update (3 DFMA)",
                # dram__bytes_read.sum + dram__bytes_write.sum of one async launch (ncu, K = 2000; the rod is
                # loaded once and the per-step exchange stays in L2, so the figure does not grow with K)
                "traffic": ASYNC_KERNEL_DRAM_BYTES,
                "traffic_source": "ncu capture of async_persistent_kernel<double,8>, K=2000 (profiles/)",
                "per_kernel": {k: {"Gupdates_per_s": v / 1e9, "frac": v / peak_upd} for k, v in per.items()}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args, S),
            "sync_updates_per_s": per["sync"], "async_updates_per_s": per["async"],
            "replay_updates_per_s": per["replay"],
            "async_blocked_updates_per_s": per["async_blocked"],
            "async_blocked": {"block_steps": h.get_opts()["halo_steps"], "delay_histogram_blocks": blocked_hist,
                              "note": "blocked asynchronous run (strips up to q-1 blocks old) on the same rod, "
                                      "timed on its own, not part of value"},
            "error": {"sync_vs_closed_form_max_abs": err_sync, "async_vs_sync_max_abs": async_vs_sync,
                      "replay_bit_identical": replay_exact, "delay_histogram": hist},
            "roofline": roofline, "clocks": clk, "e2e": e2e,
            "gpu_launches": 6 * args.steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(rod, seconds=10.0, S=S, all_cores=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

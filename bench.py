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

After the timed steps the default line also carries, untimed and on rank 0 of
a one-GPU run only: the measured fused multiply-add rates that bound the
on-chip kernels (FP64 and FP32), the blocked asynchronous run on the same rod,
the end-to-end rate through host buffers, and one sub-result per other
workload (the small rod, the streamed rod, the uneven rods, the inverse
problem), each with its updates/s, its error against the CPU oracle and its
roofline fraction.

Under torchrun each rank runs its own rod on its own GPU (independent problems,
no collective on the data path: weak scaling).  The CPU oracle arm
(``--impl reference``) times the plain C oracle on a bounded sample of the
same workload on the host cores.  The CPU oracle leg of the GPU arm (the
``cpu_baseline`` key and the error fields) runs the oracle only after the
timed region, in spawned worker processes.
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
ASYNC_KERNEL_DRAM_BYTES = 8_492_544 + 2_560
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
                   choices=["sine-mode-rod", "small-rod", "streamed-rod", "uneven-rods", "inverse-problem",
                            "fma-peak"],
                   help="sine-mode-rod (default): the sync vs async rod; streamed-rod: the 2^26-point "
                        "temporal-blocking rod; uneven-rods: 4096 rods in one batched launch; fma-peak: the "
                        "measured FP64 and FP32 fused multiply-add rates (the ALU rooflines)")
    p.add_argument("--dtype", default=None, choices=["f32", "f64"], help="streamed-rod / uneven-rods precision")
    p.add_argument("--halo", type=int, default=0, help="streamed-rod: steps per HBM pass (T)")
    p.add_argument("--r", type=float, default=0.25, help="streamed-rod: r (the sweep's values are 0.1, 0.25, 0.5)")
    p.add_argument("--rods", type=int, default=256, help="inverse-problem: rods in the batch")
    p.add_argument("--async-trace", action="store_true", help="inverse-problem: replayed asynchronous run")
    p.add_argument("--no-configs", action="store_true",
                   help="default workload: leave out the other workloads' sub-results")
    p.add_argument("--no-oracle", action="store_true", help="leave out the CPU oracle leg's error checks")
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




# ----------------------------------------------------------------------------- CPU oracle leg
#
# The only part of this file that runs the oracle.  It times the oracle as the
# CPU baseline and, after a timed GPU region has ended, recomputes the GPU's
# results from the same inputs (and from the delay traces the GPU recorded),
# in spawned worker processes: a process forked after CUDA was initialised can
# hang.


def _timed_oracle_call(job):
    import oracle
    name, args, kwargs = job
    t0 = time.perf_counter()
    out = getattr(oracle, name)(*args, **kwargs)
    return out, time.perf_counter() - t0


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def available_host_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


class OracleLeg:
    """Oracle calls submitted after a timed region; each is compared with the
    GPU result it recomputes when finish() collects it."""

    def __init__(self, processes=None):
        self.processes = processes or max(1, min(8, host_cores() - 2))
        self.pool = None
        self.pending = []  # (target dict, key, async result, compare function)

    def submit(self, target, key, name, args, kwargs=None, compare=None):
        import multiprocessing as mp
        if self.pool is None:
            self.pool = mp.get_context("spawn").Pool(self.processes)
        res = self.pool.apply_async(_timed_oracle_call, ((name, args, kwargs or {}),))
        self.pending.append((target, key, res, compare))

    def finish(self):
        for target, key, res, compare in self.pending:
            try:
                out, secs = res.get()
                entry = dict(compare(out) if compare else {})
                entry["oracle_seconds"] = secs
            except Exception as e:  # reported, never hidden
                entry = {"oracle_error": "%s: %s" % (type(e).__name__, e)}
            target[key] = entry
        self.pending = []
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None


def compare_exact(got):
    """compare function: max-abs difference and bit identity of a GPU array
    against the oracle's."""
    got = np.asarray(got)

    def cmp(ref):
        ref = np.asarray(ref)
        d = np.abs(got.astype(np.float64) - ref.astype(np.float64))
        return {"max_abs": float(d.max()) if d.size else 0.0,
                "bit_identical": bool(got.dtype == ref.dtype and np.array_equal(got, ref))}
    return cmp


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
    P = host_cores()
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


# ----------------------------------------------------------------------------- GPU arm helpers


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


_SETUP = None


def _device_setup():
    global _SETUP
    if _SETUP is not None:
        return _SETUP
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build_once(rank, world)
    _SETUP = (torch, rank, world, local)
    return _SETUP


def _max_over_ranks(torch, world, x, dev):
    from paper_1510_08982_gb300 import dist as hd
    return hd.max_over_ranks(x, world, dev)


def event_seconds(torch, stream, fn):
    """Device time of fn()'s launches on `stream` (CUDA events)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3


# ----------------------------------------------------------------------------- ALU rooflines

_ALU = None


def alu_peaks(torch, dev):
    """The two arithmetic rooflines of the on-chip kernels, in updates/s.

    measured: heat1d_probe_fma on this GPU (best of three launches, each
    ~100 ms: independent fused multiply-add chains, nothing else), divided by
    the instructions one update issues on that pipe (3: FP64 runs issue three
    DFMA; FP32 runs one FADD and two FFMA, all on the FMA pipe).
    nominal: FP64 1.25 TFLOP/s (the recipe table) = 6.25e11 DFMA/s; FP32 128
    FMA-pipe lanes per clock per SM x SMs x 2070 MHz."""
    global _ALU
    if _ALU is not None:
        return _ALU
    from paper_1510_08982_gb300 import heat1d
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    f64, shapes64 = heat1d.probe_fma("float64")
    f32, shapes32 = heat1d.probe_fma("float32")
    nom64 = FP64_NOMINAL_TFLOPS * 1e12 / 2
    nom32 = nsm * 128 * 2.07e9
    _ALU = {"f64": {"fma_per_s": f64, "updates_per_s": f64 / 3, "nominal_fma_per_s": nom64,
                    "nominal_updates_per_s": nom64 / 3, "shapes": shapes64},
            "f32": {"fma_per_s": f32, "updates_per_s": f32 / 3, "nominal_fma_per_s": nom32,
                    "nominal_updates_per_s": nom32 / 3, "shapes": shapes32},
            "source": "heat1d_probe_fma on this GPU in this run: best over 4 launch shapes of 3 timed launches "
                      "each (profiles/fma_probe_rates.md); 3 FMA-pipe instructions per update"}
    return _ALU


def alu_roofline(kernel, achieved_ups, dt, alu):
    """Roofline entry of an ALU-bound kernel: the peak derived from the unit
    counts and clocks (FP64 1.25 TFLOP/s; FP32 128 FMA lanes per SM per clock
    at 2070 MHz; 3 FMA-pipe instructions per update), with the rate measured
    by the probe on this GPU beside it.  The pure-FMA probe saturates below
    the FP64 figure (1.68 DFMA per SM per clock) and the stencil kernels
    exceed it, so the nominal figure is the bound."""
    a = alu[dt]
    return {"bound": "alu", "kernel": kernel, "achieved": achieved_ups / 1e9,
            "peak": a["nominal_updates_per_s"] / 1e9, "unit": "Gupdates/s",
            "frac": achieved_ups / a["nominal_updates_per_s"],
            "peak_source": ("nominal %s: %.3g FMA/s / 3 per update; measured on this GPU in this run: %.3g FMA/s "
                            "(%s)" % ("FP64 1.25 TFLOP/s" if dt == "f64" else "FP32 128 lanes x SMs x 2070 MHz",
                                      a["nominal_fma_per_s"], a["fma_per_s"], alu["source"])),
            "peak_measured": a["updates_per_s"] / 1e9, "frac_of_measured": achieved_ups / a["updates_per_s"]}


def run_fma_peak(args):
    torch, rank, world, local = _device_setup()
    dev = torch.device("cuda", local)
    clocks = ClockSampler(local)
    clocks.start()
    alu = alu_peaks(torch, dev)
    clk = clocks.stop()
    line = {"metric": "fused multiply-add rate (FP64 and FP32 pipes)", "value": alu["f64"]["fma_per_s"],
            "unit": "DFMA/s", "n_gpus": world, "steps": 3, "warmup": 1, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic", "config": {"workload": "heat1d_probe_fma"},
            "fma": alu, "clocks": clk, "gpu_launches": 8}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- streamed rod (config 3)


def cone_job(u0, r, c1, cN, K, i, np_dt):
    """Oracle job computing u_i(K) alone: u_i(K) depends only on
    u_{i-K..i+K}(0), so the oracle runs on the window [i-K-1, i+K+1] with its
    two ends held fixed (an error there needs K+1 steps to reach i), or the
    real Dirichlet end where the window meets it."""
    N = u0.size
    lo, hi = max(0, i - K - 1), min(N - 1, i + K + 1)
    w = np.array(u0[lo:hi + 1], dtype=np.float64)
    wc1 = c1 if lo == 0 else float(w[0])
    wcN = cN if hi == N - 1 else float(w[-1])
    return ("sync", (w, r, wc1, wcN, K), {"dtype": np_dt}), i - lo


def measure_streamed(dt, T, r, K, N, steps, warmup, leg=None, rank=0):
    """The 2^26-point rod (c1 = cN = 0, u(0) ~ U[0,1) seeded, K = 1e4)
    advanced by the streamed synchronous run, T steps per HBM pass."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    dev = torch.device("cuda", local)
    esz = 4 if dt == "f32" else 8
    tdt = torch.float32 if dt == "f32" else torch.float64
    np_dt = np.float32 if dt == "f32" else np.float64
    rod = inputs.uniform_rod(N=N, K=K, r=r, seed=hd_seed(rank))
    u0_host = rod.u0.astype(np_dt)
    u0 = torch.tensor(u0_host, device=dev)
    h = heat1d.Heat1d(N, r, 0.0, 0.0, dtype="float32" if dt == "f32" else "float64", sync_mode=2, halo_steps=T)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        h.set_u(u0)
        h.run_sync(K)
    h.sync()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    total = 0.0
    for _ in range(steps):
        h.set_u(u0)  # 2*N*esz bytes > L2: the rod itself flushes L2
        total += event_seconds(torch, stream, lambda: h.run_sync(K))
    clk = clocks.stop()
    h.sync()
    total = _max_over_ranks(torch, world, total, dev)
    samples = [1, N // 3, N // 2 + 12345, N - 2]
    if leg is not None:  # the synchronous result, sampled before the asynchronous runs reuse the handle
        got_t = h.get_u(device=True)
        got = got_t[torch.tensor(samples, device=dev)].cpu().numpy()
        mp_ok = bool(float(got_t.min()) >= 0.0 and float(got_t.max()) <= 1.0)
        del got_t
    # The asynchronous run with temporal blocking on the same tiles (Eq.
    # (eqn:async) per block of T steps, strips up to q-1 blocks old), timed
    # after the synchronous one on the same handle, free-running with its
    # trace recorded.
    btr = h.new_blocked_trace(K)
    for _ in range(max(1, min(warmup, 1))):
        h.set_u(u0)
        h.run_async_blocked(K, btr)
    h.sync()
    atotal = 0.0
    for _ in range(steps):
        h.set_u(u0)
        atotal += event_seconds(torch, stream, lambda: h.run_async_blocked(K, btr))
    h.sync()
    atotal = _max_over_ranks(torch, world, atotal, dev)
    a_hist = np.bincount(btr.cpu().numpy().reshape(-1), minlength=Q).tolist()
    secs = total / steps
    ups = world * (N - 2) * K / secs
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alu = alu_peaks(torch, dev)
    alg_bytes = 2.0 * esz * N * (K / T)  # each pass reads and writes the rod once
    achieved_gbs = alg_bytes / secs / 1e9
    alu_ups = alu[dt]["nominal_updates_per_s"]
    hbm_ups = hbm * 1e9 / (2.0 * esz / T)
    if hbm_ups < alu_ups:
        roof = {"bound": "hbm", "kernel": "stream_tma_kernel", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                "frac": achieved_gbs / hbm, "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = alu_roofline("stream_tma_kernel", ups, dt, alu)
    per_pass = STREAM_F32_DRAM_BYTES_PER_PASS.get(T) if dt == "f32" and N == 1 << 26 else None
    traffic = None if per_pass is None else per_pass * math.ceil(K / T)
    roof.update({"traffic": traffic,
                 "traffic_source": None if traffic is None else
                 "ncu dram__bytes_read+write of this kernel on this rod, per pass x passes (profiles/)",
                 "hbm_roofline_updates_per_s": hbm_ups, "alu_roofline_updates_per_s": alu_ups,
                 "algorithmic_bytes_per_update": 2.0 * esz / T, "achieved_algorithmic_GBs": achieved_gbs})
    line = {"metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt, "data": "synthetic",
            "config": {"workload": "streamed rod: N=%d %s, r=%g, c1=cN=0, u(0)~U[0,1), K=%d, T=%d steps per "
                                   "HBM pass" % (N, dt.upper(), r, K, T), "N": N, "K": K, "T": T, "r": r,
                       "l2": "inputs larger than L2 (%d MB state)" % (N * esz >> 20)},
            "roofline": roof, "clocks": clk, "gpu_launches": 2 * steps}
    a_secs = atotal / steps
    a_ups = world * (N - 2) * K / a_secs
    a_roof = {"kernel": "stream_async_kernel"}
    if roof["bound"] == "hbm":
        a_gbs = alg_bytes / a_secs / 1e9
        a_roof.update({"bound": "hbm", "achieved": a_gbs, "peak": hbm, "unit": "GB/s", "frac": a_gbs / hbm})
    else:
        a_roof.update({"bound": "alu", "achieved": a_ups / 1e9, "peak": alu_ups / 1e9, "unit": "Gupdates/s",
                       "frac": a_ups / alu_ups})
    line["async_blocked"] = {
        "updates_per_s": a_ups, "ms_per_run": a_secs * 1e3, "vs_sync": a_ups / ups, "roofline": a_roof,
        "q": Q, "delay_histogram_blocks": a_hist,
        "note": "asynchronous run with temporal blocking streamed through HBM (tiles as segments, strips "
                "up to q-1 blocks old, trace recorded), same handle and T, timed after the synchronous run; "
                "parity: tests/test_gpu_stream_async.py replays such runs in the oracle bit for bit"}
    line["gpu_launches"] += 2 * steps
    if leg is not None:
        # sampled outputs of the last timed synchronous run, each recomputed
        # by the oracle on its dependency cone
        u0f = u0_host.astype(np.float64)
        errs = {}
        line["error"] = {"maximum_principle_holds": mp_ok, "oracle_cones": errs,
                         "note": "u_i(K) at %d sampled points, each recomputed by the oracle (%s mode) on the "
                                 "2K+3-point window that determines it" % (len(samples), dt.upper())}
        for i, g in zip(samples, got):
            job, at = cone_job(u0f, r, 0.0, 0.0, K, i, np_dt)
            leg.submit(errs, "i=%d" % i, *job, compare=lambda ref, g=g, at=at: {
                "gpu": float(g), "oracle": float(ref[at]), "bit_identical": bool(g == ref[at])})
    h.close()
    return line


def run_streamed(args):
    torch, rank, world, local = _device_setup()
    dt = args.dtype or "f32"
    leg = None if args.no_oracle or rank != 0 or world != 1 else OracleLeg()
    line = measure_streamed(dt, args.halo or (128 if dt == "f32" else 32), args.r,
                            args.K if args.K != K_DEFAULT else 10_000, args.N if args.N != N_DEFAULT else 1 << 26,
                            args.steps, args.warmup, leg=leg)
    if leg is not None:
        leg.finish()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- small rod (config 1)


def measure_small(K, steps, warmup, leg=None):
    """The small rod (N = 1024 FP64, r = 0.4, c1 = 0, cN = 1, u(0) = sin(pi x) +
    0.5 sin(7 pi x) + x, S = 8, q = 3): latency-bound.  Per-step device times
    of the persistent synchronous run, the free asynchronous run, its replay,
    the asynchronous run with temporal blocking (the default block length: 32
    steps on these 128-point segments), and a synchronous run relaunched once
    per step (the paper's structure without its host copies); then async vs
    sync at equal error: the steps and the time to ||u(k) - u_ss||_inf <= 1e-6."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    dev = torch.device("cuda", local)
    rod = inputs.small_rod()
    N, S = rod.N, 8
    eps, every = 1e-6, 1024
    h = heat1d.Heat1d(N, rod.r, rod.c1, rod.cN, dtype="float64", segments=S, q=Q)
    T = h.get_opts()["halo_steps"]
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
        return event_seconds(torch, stream, fn)

    btr = h.new_blocked_trace(K)
    runs = {"sync": lambda: h.run_sync(K), "async": lambda: h.run_async(K, tr), "replay": lambda: h.replay(K, tr),
            "async_blocked": lambda: h.run_async_blocked(K, btr), "sync_relaunch_per_step": lambda: relaunch(K)}
    for _ in range(warmup):
        for f in runs.values():
            timed(f)
    h.sync()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    tot = {k: 0.0 for k in runs}
    for _ in range(steps):
        for k, f in runs.items():
            tot[k] += timed(f)
    h.sync()
    clk = clocks.stop()
    outputs = {}
    if leg is not None:  # the last timed runs' results, for the oracle leg
        for k in ("sync", "async", "async_blocked"):
            h.set_u(u0)
            runs[k]()
            h.sync()
            outputs[k] = h.get_u(device=False)
        trh, btrh = tr.cpu().numpy(), btr.cpu().numpy()
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
                                        "seconds": eq["sync"]["steps"] * tot["sync_relaunch_per_step"] / (steps * K),
                                        "note": "per-step time of the timed relaunch run x the synchronous steps"}
    us = {k: 1e6 * v / (steps * K) for k, v in tot.items()}
    upd = (N - 2) * K
    ups = {k: upd * steps / v for k, v in tot.items()}
    t_step = tot["sync"] + tot["async"] + tot["replay"]
    value = world * 3 * upd * steps / _max_over_ranks(torch, world, t_step, dev)
    alu = alu_peaks(torch, dev)
    roof = alu_roofline("async_persistent_kernel<double,2> (free run + replay)",
                        2 * upd * steps / (tot["async"] + tot["replay"]), "f64", alu)
    roof.update({"traffic": None, "note": "8 CTAs on a 1024-point rod: bound by exchange latency, the ALU "
                                          "fraction is reported but not meaningful"})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": 1e3 * t_step / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "small rod: N=1024 FP64, r=0.4, c1=0, cN=1, u(0)=sin(pi x)+0.5 sin(7 pi x)+x, "
                                   "K=%d, S=8, q=3; step = sync + async (trace recorded) + replay" % K,
                       "N": N, "K": K, "segments": S, "q": Q, "T": T,
                       "l2": "the 8 KB rod stays on-chip; latency-bound, L2 state does not matter"},
            "us_per_step": us, "updates_per_s": ups,
            "blocked_delay_histogram": np.bincount(btr.cpu().numpy().reshape(-1), minlength=Q).tolist(),
            "speedup": {"async_vs_relaunch_per_step": us["sync_relaunch_per_step"] / us["async"],
                        "async_blocked_vs_relaunch_per_step": us["sync_relaunch_per_step"] / us["async_blocked"],
                        "persistent_sync_vs_relaunch_per_step": us["sync_relaunch_per_step"] / us["sync"]},
            "equal_error": eq, "roofline": roof, "clocks": clk, "gpu_launches": steps * (4 + K)}
    if leg is not None:
        errs = {}
        line["error"] = {"oracle": errs, "note": "full runs of K=%d recomputed by the oracle (async and blocked "
                                                 "from the traces the GPU recorded)" % K}
        a = (rod.u0, rod.r, rod.c1, rod.cN)
        leg.submit(errs, "sync", "sync", a + (K,), compare=compare_exact(outputs["sync"]))
        leg.submit(errs, "async_replay", "async_replay", a + (S, Q, K, trh), compare=compare_exact(outputs["async"]))
        leg.submit(errs, "async_blocked", "async_blocked", a + (S, Q, T, K, btrh),
                   compare=compare_exact(outputs["async_blocked"]))
    h.close()
    return line


def run_small(args):
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import inputs
    K = args.K if args.K != K_DEFAULT else inputs.small_rod().K
    leg = None if args.no_oracle or rank != 0 or world != 1 else OracleLeg()
    line = measure_small(K, args.steps, args.warmup, leg=leg)
    if leg is not None:
        leg.finish()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        err = line.get("error", {}).get("oracle", {})
        secs = sum(v.get("oracle_seconds", 0.0) for v in err.values())
        if secs > 0:
            line["cpu_baseline"] = {"value": 3 * (1024 - 2) * K / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "plain C oracle, one thread per run: full synchronous run, replay of "
                                              "the recorded trace and blocked replay, K=%d (%.2f s)" % (K, secs)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- uneven rods (config 4)


def measure_uneven(dt, steps, warmup, e2e=True, leg=None):
    """4096 uneven rods in one batched persistent launch, replayed from a CUDA graph."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs, tune
    dev = torch.device("cuda", local)
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
    for _ in range(warmup):
        u.copy_(u0)
        graph.replay()
    torch.cuda.synchronize()
    b.sync()
    clocks = ClockSampler(local)
    clocks.start()
    total = 0.0
    for _ in range(steps):
        u.copy_(u0)
        flush.fill_(1.0)
        total += event_seconds(torch, stream, graph.replay)
    clk = clocks.stop()
    b.sync()
    total = _max_over_ranks(torch, world, total, dev)
    secs = total / steps
    ups = world * updates / secs
    alu = alu_peaks(torch, dev)
    got = u.cpu().numpy() if leg is not None else None  # the last timed run's result
    e2e_out = None
    if e2e:
        pinned = torch.empty(total_n, dtype=tdt).pin_memory()
        pinned.copy_(torch.tensor(host, dtype=tdt))
        out = torch.empty_like(pinned).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            u.copy_(pinned, non_blocking=True)
            b.run(u)
            out.copy_(u, non_blocking=True)
            torch.cuda.synchronize()
        dt_e2e = (time.perf_counter() - t0) / steps
        b.sync()
        e2e_out = {"value": world * updates / dt_e2e, "unit": UNIT, "h2d_bytes_per_step": total_n * esz,
                   "d2h_bytes_per_step": total_n * esz,
                   "path": "pinned host -> device, heat1d_batch_run, device -> host"}
    # The asynchronous batched run on the same batch (the parts of split
    # rods exchange strips with up to q-1 blocks of delay), free-running with
    # its trace recorded, timed after the synchronous one.
    atr = b.new_trace()
    u.copy_(u0)
    b.run_async(u, atr)
    b.sync()
    atotal = 0.0
    for _ in range(max(1, steps)):
        u.copy_(u0)
        atotal += event_seconds(torch, stream, lambda: b.run_async(u, atr))
    b.sync()
    atotal = _max_over_ranks(torch, world, atotal, dev)
    a_ups = world * updates / (atotal / max(1, steps))
    a_got = u.cpu().numpy() if leg is not None else None
    a_trace = atr.cpu().numpy()
    roof = alu_roofline("batched_kernel", ups, dt, alu)
    roof["traffic"] = None
    line = {"metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt, "data": "synthetic",
            "async": {"updates_per_s": a_ups, "vs_sync": a_ups / ups,
                      "frac": a_ups / alu[dt]["nominal_updates_per_s"], "q": Q, "T": opts.get("halo_steps"),
                      "delay_histogram_blocks": np.bincount(a_trace.reshape(-1), minlength=Q).tolist(),
                      "note": "asynchronous batched run (heat1d_batch_run_async): the parts of split rods are the "
                              "segments of the blocked model; rods on one CTA or warp run as in the synchronous "
                              "launch; timed after the synchronous replays, not part of value"},
            "config": {"workload": "uneven rods: 4096 rods, N log-U[256,65536], K log-U[1e3,1e5], r U[0.05,0.5], "
                                   "8 sine modes; one batched persistent launch replayed from a CUDA graph; tile "
                                   "and halo depth from the autotuner",
                       "rods": len(rods), "points": total_n, "updates": updates, "plan": info, "opts": opts,
                       "l2": "flushed between timed steps (256 MB write)"},
            "roofline": roof, "clocks": clk, "e2e": e2e_out, "gpu_launches": steps + 1 + max(1, steps)}
    if leg is not None:
        cheap = [j for j, r in enumerate(rods) if r.N * r.K <= 2e7]
        pick = [int(j) for j in np.random.default_rng(1).choice(cheap, size=24, replace=False)]
        heaviest = max(range(len(rods)), key=lambda j: rods[j].N * rods[j].K)
        errs = {}
        line["error"] = {"oracle": errs, "note": "24 seeded rods and the heaviest rod (N=%d, K=%d) recomputed by "
                                                 "the oracle (%s mode)" % (rods[heaviest].N, rods[heaviest].K,
                                                                           dt.upper())}
        np_dt = np.float32 if dt == "f32" else np.float64
        for j in pick + [heaviest]:
            r = rods[j]
            leg.submit(errs, "rod %d (N=%d, K=%d)" % (j, r.N, r.K), "sync", (r.u0, r.r, r.c1, r.cN, r.K),
                       {"dtype": np_dt}, compare=compare_exact(got[off[j]:off[j] + r.N]))
        # the asynchronous run: four cheap split rods replayed by the oracle's
        # split model from the recorded delays
        T = int(opts.get("halo_steps") or b.describe()["halo_steps"])
        split = [j for j in cheap if b.rod_parts(j)[0].size > 2][:4]
        aerrs = {}
        line["async"]["error"] = {"oracle": aerrs, "note": "split rods recomputed by the oracle's blocked model "
                                                           "(async_blocked_split) from the recorded part delays"}
        for j in split:
            r = rods[j]
            offs, toff = b.rod_parts(j)
            P, nb = offs.size - 1, (r.K + T - 1) // T
            parts = a_trace[toff:toff + 2 * P * nb].reshape(P, nb, 2)
            rtr = np.zeros((nb, P - 1, 2), dtype=np.uint8)
            for bnd in range(P - 1):
                rtr[:, bnd, 0] = parts[bnd, :, 1]
                rtr[:, bnd, 1] = parts[bnd + 1, :, 0]
            u0r = r.u0.astype(np_dt).astype(np.float64)
            leg.submit(aerrs, "rod %d (N=%d, K=%d, %d parts)" % (j, r.N, r.K, P), "async_blocked_split",
                       (u0r, r.r, r.c1, r.cN, offs, Q, T, r.K, rtr), {"dtype": np_dt},
                       compare=compare_exact(a_got[off[j]:off[j] + r.N]))
    b.close()
    return line


def run_uneven(args):
    torch, rank, world, local = _device_setup()
    leg = None if args.no_oracle or rank != 0 or world != 1 else OracleLeg()
    line = measure_uneven(args.dtype or "f32", args.steps, args.warmup, e2e=not args.no_e2e, leg=leg)
    if leg is not None:
        leg.finish()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- inverse problem (config 5)


def closed_form_uK(rod, K):
    """u(K) of the synchronous run from the discrete sine transform of the
    initial data (the exact solution of Eq. (eqn:sync): each sine mode m
    decays by 1 - 4 r sin^2(m pi / (2(N-1))) per step), evaluated in FP64."""
    from scipy.fft import dst, idst
    N = rod.N
    x = np.arange(N) / (N - 1)
    uss = rod.c1 + (rod.cN - rod.c1) * x
    f = (np.where(np.arange(N) == 0, rod.c1, np.where(np.arange(N) == N - 1, rod.cN, rod.u0)) - uss)[1:-1]
    lam = 1.0 - 4.0 * rod.r * np.sin(np.arange(1, N - 1) * np.pi / (2.0 * (N - 1))) ** 2
    out = uss.copy()
    out[1:-1] += idst(dst(f, type=1) * np.exp(K * np.log(np.abs(lam))) * np.sign(lam) ** (K % 2), type=1)
    return out


def measure_inverse(dt, replayed, nr, N, K, steps, warmup, leg=None, rank=0):
    """Adjoint of the inverse problem: nr rods of N = 65536, K = 2e4, smooth
    u(0), r_true ~ U[0.1, 0.45], u_obs = u(K) at r_true + N(0, 1e-4) (u(K) from
    the closed form of the synchronous run); one step = the forward pass with
    checkpoints every 128 steps + the backward pass (recompute + transposed
    stencil), giving dL/du(0) and dL/dr per rod at 0.9 r_true."""
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    dev = torch.device("cuda", local)
    tdt = torch.float32 if dt == "f32" else torch.float64
    rods = inputs.inverse_problem_rods(n_rods=nr, N=N, K=K, seed=hd_seed(rank))
    u0 = torch.tensor(np.stack([r.u0 for r in rods]), dtype=tdt, device=dev)
    rg = 0.9 * np.array([x.r for x in rods])
    c1 = np.array([x.c1 for x in rods])
    cN = np.array([x.cN for x in rods])
    S, q = 16, 3
    trace_h = np.stack([inputs.delay_trace(K, S, q, seed=j) for j in range(nr)]) if replayed else None
    trace = None if trace_h is None else torch.tensor(trace_h, device=dev)
    uobs_h = np.stack([closed_form_uK(x, K) + inputs.observation_noise(N, seed=7000 + j) for j, x in enumerate(rods)])
    uobs = torch.tensor(uobs_h, dtype=torch.float64, device=dev)

    def step():
        return heat1d.adjoint_batched(u0, uobs, rg, c1, cN, K, trace=trace, segments=S if replayed else 0,
                                      q=q, ckpt_every=128)

    for _ in range(warmup):
        step()
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(steps):
        out = step()
    torch.cuda.synchronize()
    dt_s = (time.perf_counter() - t0) / steps
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
    if dt == "f64":
        alu = alu_peaks(torch, dev)["f64"]
        peak = alu["nominal_fma_per_s"] / (3 + 3 + 4)
        roof = {"bound": "alu", "kernel": "adj_fwd_step / adj_bwd_step", "achieved": ups / 1e9,
                "peak": peak / 1e9, "unit": "Gupdates/s (forward-equivalent)", "frac": ups / peak,
                "peak_source": "nominal FP64 1.25 TFLOP/s = 6.25e11 DFMA/s / 10 FP64 instructions per forward "
                               "update over the three passes",
                "peak_measured": alu["fma_per_s"] / 10 / 1e9,
                "frac_of_measured": ups / (alu["fma_per_s"] / 10)}
    else:
        hbm = float(measured_peaks()[0].get("hbm_gbs", 6800.0)) * 1e9
        peak = hbm / 28.0
        roof = {"bound": "hbm", "kernel": "adj_fwd_step / adj_bwd_step", "achieved": ups * 28.0 / 1e9,
                "peak": hbm / 1e9, "unit": "GB/s", "frac": ups / peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs; 28 algorithmic bytes per forward update (forward 8 + "
                               "recompute 8 + backward 12)"}
    roof["traffic"] = None
    line = {"metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": dt_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dt, "data": "synthetic",
            "config": {"workload": "inverse problem: %d rods x N=%d, K=%d, checkpoints every 128 steps, %s; one step = "
                                   "forward with checkpoints + backward (recompute + adjoint); value counts forward "
                                   "updates (rods x (N-2) x K) per second of the whole gradient computation"
                                   % (nr, N, K, "replayed trace S=16 q=3" if replayed else "synchronous"),
                       "rods": nr, "N": N, "K": K, "ckpt_every": 128},
            "seconds_per_gradient": dt_s,
            "gradient": {"grad_r_first_rods": [float(x) for x in out[2][:4]],
                         "loss_first_rods": [float(x) for x in out[3][:4]]},
            "roofline": roof, "clocks": clk, "gpu_launches": None}
    if leg is not None:
        # rod 0 through the oracle's stored-trajectory FP64 adjoint (16 bytes
        # per point and step of host memory)
        need = 16 * N * (K + 1) + (2 << 30)
        avail = available_host_bytes()
        errs = {}
        line["error"] = {"oracle": errs}
        if need <= 0.7 * avail:
            g0 = out[1][0].cpu().numpy() if hasattr(out[1], "cpu") else np.asarray(out[1][0])
            gr0, l0 = float(out[2][0]), float(out[3][0])
            r0 = rods[0]

            def cmp(ref, g0=g0, gr0=gr0, l0=l0):
                L, g, gr = ref
                return {"loss_rel": abs(l0 - L) / abs(L), "grad_u0_rel_to_max": float(np.abs(g0 - g).max() /
                                                                                     np.abs(g).max()),
                        "grad_r_rel": abs(gr0 - gr) / abs(gr), "grad_r_gpu": gr0, "grad_r_oracle": gr}
            kw = {"S": S, "q": q, "trace": trace_h[0]} if replayed else {}
            leg.submit(errs, "rod 0", "adjoint", (r0.u0.astype(np.float32).astype(np.float64) if dt == "f32"
                                                  else r0.u0, float(np.float32(rg[0])) if dt == "f32" else rg[0],
                                                  r0.c1, r0.cN, K, uobs_h[0]), kw, compare=cmp)
        else:
            line["error"]["note"] = ("oracle adjoint skipped: it needs %.1f GB of host memory, %.1f GB available"
                                     % (need / 2 ** 30, avail / 2 ** 30))
    return line


def run_inverse(args):
    torch, rank, world, local = _device_setup()
    leg = None if args.no_oracle or rank != 0 or world != 1 else OracleLeg(processes=1)
    line = measure_inverse(args.dtype or "f64", args.async_trace, args.rods,
                           args.N if args.N != N_DEFAULT else 65536, args.K if args.K != K_DEFAULT else 20_000,
                           args.steps, args.warmup, leg=leg)
    if leg is not None:
        leg.finish()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- the default line (config 2)


def sub_configs(leg):
    """One compact sub-result per other workload (untimed extras of the
    default line): updates/s, the oracle check, the roofline fraction."""
    out = {}

    def keep(line, extra=()):
        d = {"workload": line["config"]["workload"], "value": line["value"], "unit": line["unit"],
             "dtype": line["dtype"], "steps": line["steps"], "warmup": line["warmup"],
             "ms_per_step": line["ms_per_step"], "roofline": line.get("roofline"), "clocks": line.get("clocks")}
        for k in extra:
            if k in line:
                d[k] = line[k]
        if "error" in line:
            d["error"] = line["error"]
        return d

    small = measure_small(10_000, 3, 3, leg=leg)
    out["small_rod"] = keep(small, ("us_per_step", "updates_per_s", "equal_error", "speedup"))
    streamed = {}
    for dt, T in (("f32", 1), ("f32", 128), ("f64", 32)):
        line = measure_streamed(dt, T, 0.25, 10_000, 1 << 26, 1 if (dt == "f64" or T == 1) else 3, 1, leg=leg)
        streamed["%s_T%d" % (dt, T)] = keep(line)
    out["streamed_rod"] = streamed
    out["uneven_rods"] = {dt: keep(measure_uneven(dt, 1 if dt == "f64" else 5, 1 if dt == "f64" else 2, e2e=False,
                                                  leg=leg))
                          for dt in ("f32", "f64")}
    inv = {}
    for dt, replayed in (("f64", False), ("f64", True), ("f32", False)):
        line = measure_inverse(dt, replayed, 256, 65536, 20_000, 1, 1, leg=leg)
        inv["%s_%s" % (dt, "replayed" if replayed else "sync")] = keep(line, ("seconds_per_gradient", "gradient"))
    out["inverse_problem"] = inv
    return out


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
    if args.workload == "fma-peak":
        return run_fma_peak(args)
    torch, rank, world, local = _device_setup()
    from paper_1510_08982_gb300 import heat1d, inputs
    from paper_1510_08982_gb300 import dist as hd
    dev = torch.device("cuda", local)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu = alu_peaks(torch, dev)  # before the timed region: ~1 s of probe launches
    rod = inputs.sine_mode_rod(N=args.N, K=args.K, seed=hd.rod_seed(rank))
    N, K = rod.N, rod.K
    M = N - 2
    h = heat1d.Heat1d(N, rod.r, rod.c1, rod.cN, dtype="float64", segments=nsm, q=Q)
    S = h.S
    T = h.get_opts()["halo_steps"]
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
    leg = OracleLeg() if (rank == 0 and world == 1 and not args.no_oracle) else None

    # --- full runs for the error fields (untimed); the oracle recomputes them --------------
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
    tr_host = trace.cpu().numpy()
    h.set_u(u0)
    h.replay(K, trace)
    h.sync()
    replay_exact = bool(np.array_equal(h.get_u(device=False), u_async))
    async_vs_sync = float(np.abs(u_async - u_sync).max())
    hist = np.bincount(tr_host.reshape(-1), minlength=Q).tolist()
    btr = h.new_blocked_trace(K)
    h.set_u(u0)
    h.run_async_blocked(K, btr)
    h.sync()
    u_blocked = h.get_u(device=False)
    btr_host = btr.cpu().numpy()
    error = {"sync_vs_closed_form_max_abs": err_sync, "async_vs_sync_max_abs": async_vs_sync,
             "replay_bit_identical": replay_exact, "delay_histogram": hist}
    if leg is not None:
        oracle_err = {}
        error["oracle"] = oracle_err
        error["oracle_note"] = ("full K=%d runs recomputed by the CPU oracle after the timed region: the "
                                "synchronous sweep, and the free asynchronous and blocked runs replayed from the "
                                "delay traces the GPU recorded" % K)
        a = (rod.u0, rod.r, rod.c1, rod.cN)
        leg.submit(oracle_err, "sync", "sync", a + (K,), compare=compare_exact(u_sync))
        leg.submit(oracle_err, "async_replay", "async_replay", a + (S, Q, K, tr_host), compare=compare_exact(u_async))
        leg.submit(oracle_err, "async_blocked", "async_blocked", a + (S, Q, T, K, btr_host),
                   compare=compare_exact(u_blocked))

    # --- the blocked asynchronous run on the same rod (its own timing, not part of the step) --
    t_blocked = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        h.set_u(u0)
        t_blocked += event_seconds(torch, stream, lambda: h.run_async_blocked(K, btr)) * 1e3
    h.sync()
    t_blocked = hd.max_over_ranks(t_blocked, world, dev)
    per["async_blocked"] = M * K / (t_blocked / args.steps * 1e-3)
    blocked_hist = np.bincount(btr.cpu().numpy().reshape(-1), minlength=Q)[:Q].tolist()

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

    # --- roofline of the dominant kernel: the asynchronous persistent kernel, both launches
    achieved = 2 * M * K / ((t_async + t_replay) / args.steps * 1e-3)
    roofline = alu_roofline("async_persistent_kernel<double,8> (free run + replay: both launches of a step)",
                            achieved, "f64", alu)
    roofline.update({
        # dram__bytes_read.sum + dram__bytes_write.sum of one async launch (ncu, K = 2000; the rod is
        # loaded once and the per-step exchange stays in L2, so the figure does not grow with K)
        "traffic": ASYNC_KERNEL_DRAM_BYTES,
        "traffic_source": "ncu capture of async_persistent_kernel<double,8>, K=2000 (profiles/)",
        "per_kernel": {k: {"Gupdates_per_s": v / 1e9, "frac": v / alu["f64"]["nominal_updates_per_s"],
                           "frac_of_measured": v / alu["f64"]["updates_per_s"]} for k, v in per.items()}})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(args, S),
            "sync_updates_per_s": per["sync"], "async_updates_per_s": per["async"],
            "replay_updates_per_s": per["replay"],
            "async_blocked_updates_per_s": per["async_blocked"],
            "async_blocked": {"block_steps": T, "delay_histogram_blocks": blocked_hist,
                              "note": "blocked asynchronous run (strips up to q-1 blocks old) on the same rod, "
                                      "timed on its own, not part of value"},
            "error": error, "roofline": roofline, "fma_rates": alu, "clocks": clk, "e2e": e2e,
            "gpu_launches": 6 * args.steps}
    if rank == 0 and world == 1 and not args.no_configs:
        line["configs"] = sub_configs(leg)
    h.close()
    if leg is not None:
        leg.finish()
        full = line["error"]["oracle"]
        line["error"]["oracle_bit_identical"] = all(v.get("bit_identical") for v in full.values())
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(rod, seconds=10.0, S=S, all_cores=True)
        if leg is not None:
            full = line["error"]["oracle"]
            secs = {k: v.get("oracle_seconds") for k, v in full.items()}
            line["cpu_baseline"]["full_workload"] = {
                "updates_per_s": {k: (M * K / s if s else None) for k, s in secs.items()},
                "seconds": secs,
                "note": "the oracle's full K runs of this line's error check, one thread each, run in parallel "
                        "worker processes"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

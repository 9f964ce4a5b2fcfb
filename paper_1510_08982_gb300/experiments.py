"""The paper's own run (Section 5), as data.

Parameters of Section 5: r = alpha*dt/dx^2 = 0.5, N = 100 grid points, one
point per PE (n = 1, so 100 segments), u_i(0) = cos^2(3 pi i / (2(N-1))),
Dirichlet ends u_1 = 1 and u_N = 0 (or the periodic ring of Section 5.3).  The
paper does not state the number of steps; 1000 is used by default.

* ``spatio_temporal`` -- Fig. 2: the state at every step of one asynchronous
  run (and of the synchronous run for comparison).
* ``ensemble`` -- Fig. 3 (Dirichlet) and Fig. 6 (periodic): ||u(k)||_2 of every
  step of 300 independent free-running asynchronous runs, their mean, the
  synchronous trajectory, and the histogram of the delays the GPU recorded.

* ``delay_statistics`` / ``decay_rates`` -- the delays the GPU recorded
  (overall and per boundary side, mean, lag-1 autocorrelation) and the
  decay rate of ||u(k) - u_ss|| from the fundamental mode, asynchronous runs
  next to the synchronous spectral radius 1 - 4 r sin^2(pi/(2(N-1))).  The companion
  paper's theory of these rates is not available here, so nothing is
  compared against a predicted value.

``python -m paper_1510_08982_gb300.experiments --out run.npz [--periodic]``
writes the arrays to an .npz file.  Every run is a run of the library (no
CPU path); each asynchronous run's trace is kept so that it can be replayed.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import heat1d, inputs

N_PAPER = 100
R_PAPER = 0.5


def _handle(periodic: bool, q: int, dtype: str):
    return heat1d.Heat1d(N_PAPER, R_PAPER, 1.0, 0.0, dtype=dtype, segments=N_PAPER, q=q,
                         boundary=1 if periodic else 0, halo_steps=1)


def spatio_temporal(K: int = 1000, q: int = 3, periodic: bool = False, dtype: str = "float64"):
    """States of every step: (async (K+1, N), sync (K+1, N), async trace)."""
    import torch
    rod = inputs.paper_rod(N=N_PAPER, K=K)
    tdt = torch.float64 if dtype == "float64" else torch.float32
    with _handle(periodic, q, dtype) as h:
        snaps = torch.empty((K + 1, N_PAPER), dtype=tdt, device="cuda")
        h.set_snapshots(snaps, every=1)
        h.set_u(rod.u0)
        tr = h.new_trace(K)
        h.run_async(K, tr)
        h.sync()
        a = snaps.cpu().numpy()
        h.set_u(rod.u0)
        h.run_sync(K)
        h.sync()
        s = snaps.cpu().numpy()
        h.set_snapshots(None)
    return a, s, tr.cpu().numpy()


def ensemble(runs: int = 300, K: int = 1000, q: int = 3, periodic: bool = False, dtype: str = "float64",
             keep_traces: bool = False):
    """||u(k)||_2 for k = 0..K of `runs` free asynchronous runs and of the
    synchronous run, plus the delay histogram over all runs."""
    import torch
    rod = inputs.paper_rod(N=N_PAPER, K=K)
    tdt = torch.float64 if dtype == "float64" else torch.float32
    norms = np.empty((runs, K + 1))
    hist = np.zeros(q, dtype=np.int64)
    traces = []
    with _handle(periodic, q, dtype) as h:
        snaps = torch.empty((K + 1, N_PAPER), dtype=tdt, device="cuda")
        h.set_snapshots(snaps, every=1)
        tr = h.new_trace(K)
        for j in range(runs):
            h.set_u(rod.u0)
            h.run_async(K, tr)
            h.sync()
            norms[j] = torch.linalg.vector_norm(snaps.double(), dim=1).cpu().numpy()
            hist += torch.bincount(tr.reshape(-1).long(), minlength=q).cpu().numpy()[:q]
            if keep_traces:
                traces.append(tr.cpu().numpy())
        h.set_u(rod.u0)
        h.run_sync(K)
        h.sync()
        sync_norm = torch.linalg.vector_norm(snaps.double(), dim=1).cpu().numpy()
        h.set_snapshots(None)
    out = {"norms": norms, "mean_norm": norms.mean(axis=0), "sync_norm": sync_norm, "delay_histogram": hist}
    if keep_traces:
        out["traces"] = np.stack(traces)
    return out


def delay_statistics(trace, q: int):
    """trace: uint8 (K, B, 2).  Histogram, mean, per-side histograms and the
    lag-1 autocorrelation of each boundary side's delay sequence (averaged)."""
    t = np.asarray(trace, dtype=np.float64)
    hist = np.bincount(np.asarray(trace).reshape(-1), minlength=q)[:q]
    per_side = [np.bincount(np.asarray(trace)[:, :, s].reshape(-1), minlength=q)[:q] for s in (0, 1)]
    x = t - t.mean(axis=0, keepdims=True)
    num = (x[1:] * x[:-1]).sum(axis=0)
    den = (x * x).sum(axis=0)
    ac = float(np.mean(num[den > 0] / den[den > 0])) if np.any(den > 0) else 0.0
    return {"histogram": hist, "mean": float(t.mean()), "per_side": np.stack(per_side), "lag1_autocorrelation": ac}


def decay_rates(K: int = 20000, runs: int = 4, q: int = 3, dtype: str = "float64"):
    """Per-step decay factor of ||u(k) - u_ss||_2 (fitted on the last half of
    the run) for `runs` asynchronous runs and the synchronous run, from the
    fundamental mode u(0) = u_ss + sin(pi x) on the Section 5 rod.  The
    synchronous factor is then lambda_1 = 1 - 4 r sin^2(pi / (2 (N - 1)))
    from the first step (the paper's own u(0) has no fundamental component,
    so its error decays through a mix of modes instead)."""
    import torch
    x = inputs.grid_x(N_PAPER)
    uss_np = 1.0 - x
    u0 = uss_np + np.sin(np.pi * x)
    uss = torch.tensor(uss_np, dtype=torch.float64, device="cuda")
    tdt = torch.float64 if dtype == "float64" else torch.float32
    every = max(1, K // 2000)
    rows = K // every + 1

    def rate(snaps):
        e = torch.linalg.vector_norm(snaps.double() - uss, dim=1).cpu().numpy()
        k = np.arange(rows) * every
        half = rows // 2
        good = e[half:] > 0
        slope = np.polyfit(k[half:][good], np.log(e[half:][good]), 1)[0]
        return float(np.exp(slope))

    rates = []
    with _handle(False, q, dtype) as h:
        snaps = torch.empty((rows, N_PAPER), dtype=tdt, device="cuda")
        h.set_snapshots(snaps, every=every)
        for _ in range(runs):
            h.set_u(u0)
            h.run_async(K)
            h.sync()
            rates.append(rate(snaps))
        h.set_u(u0)
        h.run_sync(K)
        h.sync()
        sync_rate = rate(snaps)
        h.set_snapshots(None)
    lam1 = 1.0 - 4.0 * R_PAPER * np.sin(np.pi / (2.0 * (N_PAPER - 1))) ** 2
    return {"async_rates": np.array(rates), "sync_rate": sync_rate, "sync_spectral_radius": lam1}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--out", required=True)
    p.add_argument("--K", type=int, default=1000)
    p.add_argument("--runs", type=int, default=300)
    p.add_argument("--q", type=int, default=3)
    p.add_argument("--periodic", action="store_true")
    args = p.parse_args(argv)
    a, s, tr = spatio_temporal(args.K, args.q, args.periodic)
    ens = ensemble(args.runs, args.K, args.q, args.periodic)
    stats = delay_statistics(tr, args.q)
    extra = {}
    if not args.periodic:
        dr = decay_rates(q=args.q)
        extra = {"async_decay_rates": dr["async_rates"], "sync_decay_rate": dr["sync_rate"],
                 "sync_spectral_radius": dr["sync_spectral_radius"]}
    np.savez_compressed(args.out, async_states=a, sync_states=s, async_trace=tr,
                        delay_mean=stats["mean"], delay_per_side=stats["per_side"],
                        delay_lag1_autocorrelation=stats["lag1_autocorrelation"], **ens, **extra)
    print("wrote %s: %d runs x %d steps, delay histogram %s, mean delay %.3f, lag-1 autocorrelation %.3f%s"
          % (args.out, args.runs, args.K, ens["delay_histogram"].tolist(), stats["mean"],
             stats["lag1_autocorrelation"],
             "" if args.periodic else ", decay per step: sync %.6f (lambda_1 %.6f), async %s"
             % (extra["sync_decay_rate"], extra["sync_spectral_radius"],
                np.round(extra["async_decay_rates"], 6).tolist())))


if __name__ == "__main__":
    main()

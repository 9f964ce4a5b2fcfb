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
    np.savez_compressed(args.out, async_states=a, sync_states=s, async_trace=tr, **ens)
    print("wrote %s: %d runs x %d steps, delay histogram %s" % (args.out, args.runs, args.K,
                                                                ens["delay_histogram"].tolist()))


if __name__ == "__main__":
    main()

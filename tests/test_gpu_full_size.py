"""GPU parity at the workloads' full sizes, against the CPU oracle.

- Sync vs async at scale: the 2^20-point FP64 rod (r = 0.25, ends -1 and 1,
  16 sine modes), one segment per SM, q = 3, the full K = 1e5 steps in the
  benchmark's launch configuration.  The synchronous run is compared with the
  oracle's sweep (Section 2, Eq. (eqn:sync)); the free asynchronous run and the
  free blocked asynchronous run are replayed by the oracle from the delay
  traces the GPU recorded (Section 3, Eq. (eqn:async), and its blocked
  reading).  All three must agree bit for bit (and within 1e-12).  The three
  oracle runs (about 1e11 updates each) run in parallel worker processes.
- Inverse problem: one rod of N = 65536, K = 2e4, checkpoints every 128 steps,
  FP64, synchronous and replayed (S = 16, q = 3, seeded delays): the loss,
  dL/du(0) and dL/dr of the GPU adjoint against the oracle's stored-trajectory
  adjoint, and directional central differences at h = 1e-6 of oracle forward
  runs.  The oracle stores the whole trajectory and its adjoint (16 bytes per
  point and step, 21 GB at this size); on a host with less memory available
  the test takes the largest K that fits and says so.
"""
from __future__ import annotations

import warnings

import numpy as np
import pytest

from paper_1510_08982_gb300 import inputs
from tests import oracle_pool

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def H():
    import torch  # noqa: F401
    from paper_1510_08982_gb300 import build, heat1d
    build.build()
    return heat1d


def assert_same(got, ref, what):
    assert got.dtype == ref.dtype, what
    err = float(np.abs(got.astype(np.float64) - ref.astype(np.float64)).max())
    assert err <= TOL64, (what, err)
    assert np.array_equal(got, ref), "%s: not bit-identical (max err %g)" % (what, err)


def test_sine_mode_rod_full_horizon_against_oracle(H):
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    rod = inputs.sine_mode_rod()                     # N = 2^20, K = 1e5
    q = 3
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype="float64", segments=nsm, q=q) as h:
        S = h.S
        T = h.get_opts()["halo_steps"]
        h.set_u(rod.u0)
        h.run_sync(rod.K)
        h.sync()
        u_sync = h.get_u(device=False)
        tr = h.new_trace(rod.K)
        h.set_u(rod.u0)
        h.run_async(rod.K, tr)
        h.sync()
        u_async = h.get_u(device=False)
        btr = h.new_blocked_trace(rod.K)
        h.set_u(rod.u0)
        h.run_async_blocked(rod.K, btr)
        h.sync()
        u_blocked = h.get_u(device=False)
        trh, btrh = tr.cpu().numpy(), btr.cpu().numpy()
    assert S == nsm and trh.max() < q and btrh.max() < q
    args = (rod.u0, rod.r, rod.c1, rod.cN)
    ref_sync, ref_async, ref_blocked = oracle_pool.run([
        ("sync", args + (rod.K,), {}),
        ("async_replay", args + (S, q, rod.K, trh), {}),
        ("async_blocked", args + (S, q, T, rod.K, btrh), {}),
    ])
    assert_same(u_sync, ref_sync, "sync")
    assert_same(u_async, ref_async, "async replayed by the oracle")
    assert_same(u_blocked, ref_blocked, "blocked async replayed by the oracle")


def _inverse_K(N, K_full):
    need = lambda K: 16 * N * (K + 1) + (1 << 30)  # noqa: E731  (trajectory + adjoint history, 1 GB slack)
    avail = oracle_pool.available_host_bytes()
    if need(K_full) <= 0.8 * avail:
        return K_full
    K = max(128, int(0.8 * avail - (1 << 30)) // (16 * N) - 1)
    warnings.warn("inverse-problem oracle adjoint at K=%d instead of %d: %.1f GB of host memory available"
                  % (K, K_full, avail / 2 ** 30))
    return K


@pytest.mark.parametrize("replayed", [False, True], ids=["sync", "replayed"])
def test_inverse_problem_full_size_adjoint_against_oracle(H, replayed):
    import torch
    rod = inputs.inverse_problem_rods(n_rods=1, seed=3)[0]      # N = 65536, K = 2e4
    N, K = rod.N, _inverse_K(rod.N, rod.K)
    S, q, C = 16, 3, 128
    trace = inputs.delay_trace(K, S, q, seed=11) if replayed else None
    args_true = (rod.u0, rod.r, rod.c1, rod.cN)
    # observations from the oracle at r_true plus N(0, 1e-4) noise; the
    # gradient is taken at 0.9 r_true
    fwd = ("async_replay", args_true + (S, q, K, trace), {}) if replayed else ("sync", args_true + (K,), {})
    uobs = oracle_pool.run([fwd])[0] + inputs.observation_noise(N, seed=9)
    r = 0.9 * rod.r
    opts = {"segments": S, "q": q} if replayed else {}
    with H.Heat1d(N, r, rod.c1, rod.cN, dtype="float64", **opts) as h:
        h.set_u(rod.u0)
        loss, g, gr = h.adjoint(K, torch.tensor(uobs), trace=trace, ckpt_every=C)
        g = g.cpu().numpy()

    hh = 1e-6
    v = np.random.default_rng(2).standard_normal(N)
    v[0] = v[-1] = 0.0

    def fwd_job(u0, rr):
        a = (u0, rr, rod.c1, rod.cN)
        return ("async_replay", a + (S, q, K, trace), {}) if replayed else ("sync", a + (K,), {})

    # the oracle adjoint alone (its memory) first, then the four FD forward runs in parallel
    L_ref, g_ref, gr_ref = oracle_pool.run([("adjoint", (rod.u0, r, rod.c1, rod.cN, K, uobs),
                                             {"S": S, "q": q, "trace": trace} if replayed else {})])[0]
    outs = oracle_pool.run([fwd_job(rod.u0 + hh * v, r), fwd_job(rod.u0 - hh * v, r),
                            fwd_job(rod.u0, r + hh), fwd_job(rod.u0, r - hh), fwd_job(rod.u0, r)])
    Ls = [0.5 * float(np.sum((u - uobs) ** 2)) for u in outs[:4]]
    fd_u = (Ls[0] - Ls[1]) / (2 * hh)
    fd_r = (Ls[2] - Ls[3]) / (2 * hh)
    # Rounding bound for dL/du(0): each backward step rounds every lambda a
    # few times (the GPU's two additions and one fused multiply-add, or the
    # oracle's three products and additions: at most 5 eps max|lambda| per
    # step, r <= 1/2), and the transposed step of Eq. (eqn:sync) has
    # nonnegative weights (1-2r, r, r) summing to at most 1, so it grows no
    # error in the max norm and max|lambda(k)| <= max|lambda(K)|: after K steps
    # each side is within 5 K eps max|lambda(K)| of the exact adjoint, the two
    # within twice that.  The replayed run is held to the same figure (there a
    # delayed read adds its weight to an earlier level, so it is a scale, not a
    # proof).
    lam_K = float(np.abs((outs[4] - uobs)[1:-1]).max())
    tol_g = 10 * K * np.finfo(np.float64).eps * lam_K
    errs = {"loss_rel": abs(loss - L_ref) / abs(L_ref), "grad_u0_max_abs": float(np.abs(g - g_ref).max()),
            "grad_u0_tol": tol_g, "grad_r_rel": abs(gr - gr_ref) / abs(gr_ref),
            "fd_u_abs": abs(fd_u - g @ v), "fd_r_abs": abs(fd_r - gr), "grad_r": gr, "K": K}
    print("inverse problem full size (%s):" % ("replayed" if replayed else "sync"), errs)
    assert errs["loss_rel"] <= 1e-13
    assert errs["grad_u0_max_abs"] <= tol_g
    assert errs["grad_r_rel"] <= 1e-11
    assert g[0] == 0.0 and g[-1] == 0.0
    assert errs["fd_u_abs"] <= 1e-6 * max(1.0, abs(fd_u))
    assert errs["fd_r_abs"] <= 1e-6 * max(1.0, abs(fd_r))

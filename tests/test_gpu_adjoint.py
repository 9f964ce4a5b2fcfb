"""GPU adjoint (checkpoint + recompute + transposed stencil through the trace)
against the oracle's FP64 adjoint, central finite differences, and itself
across checkpoint intervals; plus the torch.autograd.Function.

Tolerances: the adjoint sums in a different order from the oracle, so
grad_u0 is compared within 1e-12 of its largest entry and dL/dr within a
relative 1e-11; the loss within a relative 1e-13.  Checkpoint intervals do not
change the arithmetic, so results for different C are identical bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch  # noqa: F401
    from paper_1510_08982_gb300 import build, heat1d
    build.build()
    return heat1d


def problem(N, K, seed, r=0.3, c1=0.2, cN=-0.4):
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-1, 1, size=N)
    uobs = rng.uniform(-1, 1, size=N)
    return inputs.Rod(N=N, K=K, r=r, c1=c1, cN=cN, u0=u0), uobs


def gpu_adjoint(H, rod, uobs, S=None, q=3, trace=None, C=0, dtype="float64"):
    import torch
    opts = {"q": q}
    if S:
        opts["segments"] = S
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, dtype=dtype, **opts) as h:
        h.set_u(rod.u0)
        loss, g, gr = h.adjoint(rod.K, torch.tensor(uobs), trace=trace, ckpt_every=C)
        uK = h.get_u(device=False)
    return loss, g.cpu().numpy(), gr, uK


def close(got, ref, rel):
    scale = max(np.abs(ref).max(), 1e-300)
    return np.abs(got - ref).max() <= rel * scale


@pytest.mark.parametrize("C", [1, 7, 128, 600])
def test_sync_adjoint_matches_oracle(H, C):
    rod, uobs = problem(1000, 600, 0)
    loss, g, gr, uK = gpu_adjoint(H, rod, uobs, C=C)
    L, gref, grref = oracle.adjoint(rod.u0, rod.r, rod.c1, rod.cN, rod.K, uobs)
    assert np.array_equal(uK, oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K))
    assert abs(loss - L) <= 1e-13 * abs(L)
    assert close(g, gref, 1e-12)
    assert abs(gr - grref) <= 1e-11 * abs(grref)
    assert g[0] == 0.0 and g[-1] == 0.0


def test_adjoint_is_independent_of_checkpoint_interval(H):
    rod, uobs = problem(700, 333, 1)
    tr = inputs.delay_trace(rod.K, 5, 3, seed=4)
    outs = [gpu_adjoint(H, rod, uobs, S=5, trace=tr, C=C) for C in (1, 10, 64, 333)]
    for o in outs[1:]:
        assert o[0] == outs[0][0] and o[2] == outs[0][2] and np.array_equal(o[1], outs[0][1])


@pytest.mark.parametrize("N,S,q,K,seed", [(1000, 8, 3, 500, 0), (300, 7, 2, 400, 1), (64, 16, 4, 300, 2),
                                          (12, 12, 3, 200, 3), (5, 5, 2, 50, 4)])
def test_replay_adjoint_matches_oracle(H, N, S, q, K, seed):
    rod, uobs = problem(N, K, seed, r=0.45)
    tr = inputs.delay_trace(K, S, q, seed=seed)
    loss, g, gr, uK = gpu_adjoint(H, rod, uobs, S=S, q=q, trace=tr, C=37)
    L, gref, grref = oracle.adjoint(rod.u0, rod.r, rod.c1, rod.cN, K, uobs, S, q, tr)
    assert np.array_equal(uK, oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, q, K, tr))
    assert abs(loss - L) <= 1e-13 * abs(L)
    assert close(g, gref, 1e-12)
    assert abs(gr - grref) <= 1e-11 * abs(grref)


def test_adjoint_of_a_free_asynchronous_run(H):
    """Differentiate what the GPU actually ran: its recorded trace."""
    rod, uobs = problem(2048, 800, 5)
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN, segments=8, q=3) as h:
        h.set_u(rod.u0)
        tr = h.new_trace(rod.K)
        h.run_async(rod.K, tr)
        h.sync()
        trh = tr.cpu().numpy()
    loss, g, gr, _ = gpu_adjoint(H, rod, uobs, S=8, q=3, trace=trh, C=128)
    L, gref, grref = oracle.adjoint(rod.u0, rod.r, rod.c1, rod.cN, rod.K, uobs, 8, 3, trh)
    assert abs(loss - L) <= 1e-13 * abs(L)
    assert close(g, gref, 1e-12)
    assert abs(gr - grref) <= 1e-11 * abs(grref)


def test_adjoint_central_differences_full_size_rod(H):
    """Inverse-problem rod size (N = 65536, smooth u(0), r_true in [0.1, 0.45],
    u_obs = u(K) + N(0, 1e-4) noise), K = 2000, C = 128: directional central
    differences at h = 1e-6 in FP64 of GPU forward runs against the adjoint."""
    import torch
    rod = inputs.inverse_problem_rods(n_rods=1, K=2000, seed=3)[0]
    with H.Heat1d(rod.N, rod.r, rod.c1, rod.cN) as h:
        h.set_u(rod.u0)
        h.run_sync(rod.K)
        h.sync()
        uobs = h.get_u(device=False) + inputs.observation_noise(rod.N, seed=9)
        r_obs = rod.r
        rod_guess = inputs.Rod(N=rod.N, K=rod.K, r=r_obs * 0.9, c1=rod.c1, cN=rod.cN, u0=rod.u0)
    loss, g, gr, _ = gpu_adjoint(H, rod_guess, uobs, C=128)

    def L(u0, r):
        with H.Heat1d(rod.N, r, rod.c1, rod.cN) as h:
            h.set_u(u0)
            h.run_sync(rod.K)
            h.sync()
            uk = h.get_u(device=False)
        return 0.5 * float(np.sum((uk - uobs) ** 2))

    hh = 1e-6
    v = np.random.default_rng(2).standard_normal(rod.N)
    v[0] = v[-1] = 0.0
    fd = (L(rod_guess.u0 + hh * v, rod_guess.r) - L(rod_guess.u0 - hh * v, rod_guess.r)) / (2 * hh)
    assert abs(fd - g @ v) <= 1e-6 * max(1.0, abs(fd))
    fdr = (L(rod_guess.u0, rod_guess.r + hh) - L(rod_guess.u0, rod_guess.r - hh)) / (2 * hh)
    assert abs(fdr - gr) <= 1e-6 * max(1.0, abs(fdr))
    assert abs(L(rod_guess.u0, rod_guess.r) - loss) <= 1e-12 * loss


@pytest.mark.parametrize("N,K,C", [(1024, 400, 50), (4096, 2000, 128)])
def test_fp32_adjoint_close_to_fp64_oracle(H, N, K, C):
    """An FP32 run steps u and lambda in FP32 (the dL/dr products of a warp's
    points in one block summed in FP32, those sums in FP64).  Each step rounds lambda once more, so
    its error grows like sqrt(K) FP32 roundings: dL/du(0) is held to
    4 sqrt(K) 2^-24 of its largest entry, dL/dr to 1e-4 (relative), both
    against the FP64 oracle on the FP32-rounded inputs."""
    rod, uobs = problem(N, K, 7)
    loss, g, gr, _ = gpu_adjoint(H, rod, uobs, C=C, dtype="float32")
    r32 = float(np.float32(rod.r))
    L, gref, grref = oracle.adjoint(rod.u0.astype(np.float32).astype(np.float64), r32, np.float32(rod.c1),
                                    np.float32(rod.cN), rod.K, uobs)
    assert abs(loss - L) <= 1e-5 * abs(L)
    assert close(g, gref, 4 * np.sqrt(K) * 2.0 ** -24)
    assert abs(gr - grref) <= 1e-4 * abs(grref)


def test_fp32_replay_adjoint_close_to_fp64_oracle(H):
    """The FP32 adjoint through a replayed asynchronous run (delayed reads,
    parked contributions), with the tolerances of the synchronous FP32 test;
    the result does not depend on the checkpoint interval."""
    rod, uobs = problem(2048, 300, 9, r=0.45)
    S, q = 6, 3
    tr = inputs.delay_trace(rod.K, S, q, seed=21)
    outs = [gpu_adjoint(H, rod, uobs, S=S, q=q, trace=tr, C=C, dtype="float32") for C in (64, 1, 300)]
    loss, g, gr, _ = outs[0]
    for o in outs[1:]:
        assert o[0] == loss and o[2] == gr and np.array_equal(o[1], g)
    r32 = float(np.float32(rod.r))
    L, gref, grref = oracle.adjoint(rod.u0.astype(np.float32).astype(np.float64), r32, np.float32(rod.c1),
                                    np.float32(rod.cN), rod.K, uobs, S, q, tr)
    assert abs(loss - L) <= 1e-5 * abs(L)
    assert close(g, gref, 4 * np.sqrt(rod.K) * 2.0 ** -24)
    assert abs(gr - grref) <= 1e-4 * abs(grref)


@pytest.mark.parametrize("async_run", [False, True])
def test_batched_adjoint_matches_oracle(H, async_run):
    import torch
    nrods, N, K, S, q = 4, 2048, 300, 6, 3
    rng = np.random.default_rng(12)
    u0 = rng.uniform(-1, 1, size=(nrods, N))
    uobs = rng.uniform(-1, 1, size=(nrods, N))
    r = rng.uniform(0.1, 0.45, size=nrods)
    c1 = rng.uniform(-1, 1, size=nrods)
    cN = rng.uniform(-1, 1, size=nrods)
    traces = np.stack([inputs.delay_trace(K, S, q, seed=40 + j) for j in range(nrods)]) if async_run else None
    tr_t = torch.tensor(traces, device="cuda") if async_run else None
    uK, g, gr, ls = H.adjoint_batched(torch.tensor(u0, device="cuda"), torch.tensor(uobs, device="cuda"), r, c1, cN,
                                      K, trace=tr_t, segments=S if async_run else 0, q=q, ckpt_every=64)
    g = g.cpu().numpy()
    uK = uK.cpu().numpy()
    for j in range(nrods):
        if async_run:
            L, gref, grref = oracle.adjoint(u0[j], r[j], c1[j], cN[j], K, uobs[j], S, q, traces[j])
            uref = oracle.async_replay(u0[j], r[j], c1[j], cN[j], S, q, K, traces[j])
        else:
            L, gref, grref = oracle.adjoint(u0[j], r[j], c1[j], cN[j], K, uobs[j])
            uref = oracle.sync(u0[j], r[j], c1[j], cN[j], K)
        assert np.array_equal(uK[j], uref)
        assert abs(ls[j] - L) <= 1e-13 * abs(L)
        assert close(g[j], gref, 1e-12)
        assert abs(gr[j] - grref) <= 1e-11 * abs(grref)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("N,S", [(4096, 1024), (1024, 1024), (2052, 513)])
def test_replay_adjoint_short_segments(H, dtype, N, S):
    """Replays with segments of 4, 1 and about 4 points: every block holds far
    more segment-boundary points than threads, and one-point segments are
    both a first and a last point."""
    rod, uobs = problem(N, 120, 17, r=0.4)
    q = 3
    tr = inputs.delay_trace(rod.K, S, q, seed=23)
    loss, g, gr, uK = gpu_adjoint(H, rod, uobs, S=S, q=q, trace=tr, C=40, dtype=dtype)
    if dtype == "float64":
        L, gref, grref = oracle.adjoint(rod.u0, rod.r, rod.c1, rod.cN, rod.K, uobs, S, q, tr)
        assert np.array_equal(uK, oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, S, q, rod.K, tr))
        assert abs(loss - L) <= 1e-13 * abs(L)
        assert close(g, gref, 1e-12)
        assert abs(gr - grref) <= 1e-11 * abs(grref)
    else:
        f = np.float32
        r32, c132, cN32 = float(f(rod.r)), float(f(rod.c1)), float(f(rod.cN))
        u64 = rod.u0.astype(f).astype(np.float64)
        L, gref, grref = oracle.adjoint(u64, r32, c132, cN32, rod.K, uobs, S, q, tr)
        assert np.array_equal(uK, oracle.async_replay(u64, r32, c132, cN32, S, q, rod.K, tr, dtype=f))
        assert abs(loss - L) <= 1e-5 * abs(L)
        assert close(g, gref, 4 * np.sqrt(rod.K) * 2.0 ** -24)
        assert abs(gr - grref) <= 1e-4 * abs(grref)


@pytest.mark.parametrize("async_run", [False, True])
def test_batched_adjoint_fp32(H, async_run):
    """The batched FP32 adjoint (rod lengths a multiple of 4, so the 16-byte
    vector kernels run): u(K) bit for bit against the oracle's FP32 run, the
    gradients within the FP32 tolerances against the FP64 oracle on the
    FP32-rounded inputs."""
    import torch
    nrods, N, K, S, q = 3, 4096, 256, 8, 3
    rng = np.random.default_rng(31)
    u0 = rng.uniform(-1, 1, size=(nrods, N)).astype(np.float32)
    uobs = rng.uniform(-1, 1, size=(nrods, N))
    r = rng.uniform(0.1, 0.45, size=nrods)
    c1 = rng.uniform(-1, 1, size=nrods)
    cN = rng.uniform(-1, 1, size=nrods)
    traces = np.stack([inputs.delay_trace(K, S, q, seed=50 + j) for j in range(nrods)]) if async_run else None
    tr_t = torch.tensor(traces, device="cuda") if async_run else None
    uK, g, gr, ls = H.adjoint_batched(torch.tensor(u0, device="cuda"), torch.tensor(uobs, device="cuda"), r, c1, cN,
                                      K, trace=tr_t, segments=S if async_run else 0, q=q, ckpt_every=64)
    g = g.cpu().numpy()
    uK = uK.cpu().numpy()
    for j in range(nrods):
        r32, c132, cN32 = (float(np.float32(x)) for x in (r[j], c1[j], cN[j]))
        u64 = u0[j].astype(np.float64)
        if async_run:
            uref = oracle.async_replay(u64, r32, c132, cN32, S, q, K, traces[j], dtype=np.float32)
            L, gref, grref = oracle.adjoint(u64, r32, c132, cN32, K, uobs[j], S, q, traces[j])
        else:
            uref = oracle.sync(u64, r32, c132, cN32, K, dtype=np.float32)
            L, gref, grref = oracle.adjoint(u64, r32, c132, cN32, K, uobs[j])
        assert np.array_equal(uK[j], uref)
        assert abs(ls[j] - L) <= 1e-5 * abs(L)
        assert close(g[j], gref, 4 * np.sqrt(K) * 2.0 ** -24)
        assert abs(gr[j] - grref) <= 1e-4 * abs(grref)


def test_autograd_function(H):
    import torch
    from paper_1510_08982_gb300.autograd import heat1d_run
    rod, uobs = problem(512, 250, 8)
    u0 = torch.tensor(rod.u0, device="cuda", requires_grad=True)
    r = torch.tensor(rod.r, dtype=torch.float64, device="cuda", requires_grad=True)
    uK = heat1d_run(u0, r, rod.K, rod.c1, rod.cN, ckpt_every=32)
    loss = 0.5 * ((uK - torch.tensor(uobs, device="cuda")) ** 2).sum()
    loss.backward()
    L, gref, grref = oracle.adjoint(rod.u0, rod.r, rod.c1, rod.cN, rod.K, uobs)
    assert abs(float(loss) - L) <= 1e-13 * abs(L)
    assert close(u0.grad.cpu().numpy(), gref, 1e-12)
    assert abs(float(r.grad) - grref) <= 1e-11 * abs(grref)

"""Pins of the CPU oracle to what the paper and the mathematics fix.

Every test here runs on the CPU.  The oracle is compared with closed forms,
exact rational brute force and invariants written independently in
tests/pins.py, chosen so that a dropped term, a wrong sign, a swapped delay
side or an off-by-one in time fails at least one of them.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs
from tests import pins

EPS64 = np.finfo(np.float64).eps
HERE = os.path.dirname(os.path.abspath(__file__))


# --------------------------------------------------------------------------- golden


def read_golden(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip()
    return vals


def test_golden_paper_section5_parameters():
    """Section 5 prints dx = 0.1, dt = 0.01, alpha = 0.5 and r = alpha dt/dx^2 = 0.5,
    the cos^2 initial condition and the ends 1 and 0."""
    g = read_golden("paper_section5_parameters.txt")
    dx, dt, alpha = float(g["dx"]), float(g["dt"]), float(g["alpha"])
    assert abs(alpha * dt / dx ** 2 - float(g["r"])) < 1e-12
    rod = inputs.paper_rod(N=int(g["N"]))
    # the coded (0-based) initial condition agrees with the boundary values
    assert abs(rod.u0[0] - float(g["c1"])) < 1e-15
    assert abs(rod.u0[-1] - float(g["c2"])) < 1e-15
    assert rod.r == float(g["r"])


# --------------------------------------------------------------------------- segments


@pytest.mark.parametrize("N,S", [(10, 3), (1024, 8), (1 << 20, 148), (1 << 20, 152), (7, 7), (100, 100)])
def test_segments_rule(N, S):
    off = oracle.segments(N, S)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == N
    assert sizes.sum() == N
    extra = N % S
    assert np.all(sizes[:extra] == N // S + 1)
    assert np.all(sizes[extra:] == N // S)


# --------------------------------------------------------------------------- sync


@pytest.mark.parametrize("N,m,r,K", [(64, 1, 0.5, 500), (257, 3, 0.25, 2000), (1024, 7, 0.4, 3000),
                                     (33, 31, 0.45, 200), (100, 5, 0.1, 1000)])
def test_sync_single_mode_decay(N, m, r, K):
    """A single sine mode decays exactly by lambda_m^K (Section 2 update,
    Dirichlet 0 ends).  A sign error or a missing factor 2 fails this."""
    x = inputs.grid_x(N)
    u0 = np.sin(m * math.pi * x)
    u0[0] = 0.0
    u0[-1] = 0.0
    lam = 1.0 - 4.0 * r * math.sin(m * math.pi / (2.0 * (N - 1))) ** 2
    expect = lam ** K * u0
    got = oracle.sync(u0, r, 0.0, 0.0, K)
    tol = 4.0 * K * EPS64 * np.abs(u0).max() + 1e-15
    assert np.abs(got - expect).max() <= tol


def test_sync_small_rod_closed_form():
    """The small plain-method rod (N=1024, r=0.4, K=1e4): u(K) =
    lam_1^K sin(pi x) + 0.5 lam_7^K sin(7 pi x) + x, within the rounding bound
    4 K eps max|u|."""
    rod = inputs.small_rod()
    got = oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K)
    x = inputs.grid_x(rod.N)
    l1 = 1 - 4 * rod.r * math.sin(math.pi / (2 * (rod.N - 1))) ** 2
    l7 = 1 - 4 * rod.r * math.sin(7 * math.pi / (2 * (rod.N - 1))) ** 2
    expect = l1 ** rod.K * np.sin(math.pi * x) + 0.5 * l7 ** rod.K * np.sin(7 * math.pi * x) + x
    tol = 4.0 * rod.K * EPS64 * 2.0
    assert np.abs(got - expect).max() <= tol
    # and the general DST-based closed form agrees
    cf = pins.closed_form_sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K)
    assert np.abs(got - cf).max() <= tol


@pytest.mark.parametrize("seed", [0, 1])
def test_sync_sine_sum_closed_form_with_boundary_layer(seed):
    """Sum of sine modes with c1 = -1, cN = 1 forced at the ends (a boundary
    layer): the DST closed form of u(0) - u_ss on the interior."""
    rod = inputs.sine_mode_rod(N=4096, K=3000, seed=seed, m_max=512)
    got = oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K)
    cf = pins.closed_form_sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K)
    amp = np.abs(pins.forced(rod.u0, rod.c1, rod.cN)).max()
    assert np.abs(got - cf).max() <= 4.0 * rod.K * EPS64 * amp + 1e-12


@pytest.mark.parametrize("N,r,K", [(5, Fraction(1, 4), 20), (8, Fraction(1, 2), 20), (16, Fraction(1, 4), 20),
                                   (33, Fraction(3, 8), 12), (64, Fraction(1, 4), 18)])
def test_sync_brute_force_exact(N, r, K):
    """Dyadic data and dyadic r keep every FP64 operation exact for these K,
    so the oracle must equal A^K u(0) in rational arithmetic bit for bit."""
    rng = np.random.default_rng(N)
    u0 = rng.integers(-16, 17, size=N) / 16.0
    c1, cN = 0.5, -1.25
    exact = pins.brute_sync_fraction(u0, r, c1, cN, K)
    got = oracle.sync(u0, float(r), c1, cN, K)
    assert [Fraction(v) for v in got] == exact


def test_sync_brute_force_inexact_bound():
    """Non-dyadic r: oracle within rounding of the exact rational result."""
    N, K, r = 24, 60, Fraction(1, 3)
    rng = np.random.default_rng(5)
    u0 = rng.random(N)
    exact = np.array([float(v) for v in pins.brute_sync_fraction(u0, r, 0.3, 0.7, K)])
    got = oracle.sync(u0, float(r), 0.3, 0.7, K)
    assert np.abs(got - exact).max() <= 4 * K * EPS64


@pytest.mark.parametrize("r", [0.1, 0.25, 0.5])
def test_sync_maximum_principle(r):
    """For 0 < r <= 1/2 each update is a convex combination: every u(k) stays
    inside [min, max] of u(0) and the ends."""
    rng = np.random.default_rng(11)
    N = 777
    u0 = rng.uniform(-3, 2, size=N)
    c1, cN = 1.5, -0.5
    lo = min(u0[1:-1].min(), c1, cN)
    hi = max(u0[1:-1].max(), c1, cN)
    for K in (1, 10, 500):
        u = oracle.sync(u0, r, c1, cN, K)
        assert u.min() >= lo - 4 * EPS64 * K and u.max() <= hi + 4 * EPS64 * K


def test_sync_linear_steady_state():
    """Small N, large K: the unique steady state is the line from c1 to cN."""
    N = 16
    u0 = np.random.default_rng(2).random(N)
    u = oracle.sync(u0, 0.45, -2.0, 3.0, 20000)
    x = inputs.grid_x(N)
    assert np.abs(u - (-2.0 + 5.0 * x)).max() < 1e-12


def test_sync_fp32_mode_is_float_arithmetic():
    """The FP32 mode runs the same expression in float: on dyadic data that is
    exact in float it equals the FP64 result, elsewhere it is within the
    float rounding bound of FP64."""
    N, K = 32, 8
    rng = np.random.default_rng(3)
    u0 = rng.integers(-8, 9, size=N) / 8.0
    a = oracle.sync(u0, 0.25, 0.0, 1.0, K, dtype=np.float32)
    b = oracle.sync(u0, 0.25, 0.0, 1.0, K)
    assert a.dtype == np.float32 and np.array_equal(a.astype(np.float64), b)
    rod = inputs.small_rod(K=2000)
    a = oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K, dtype=np.float32).astype(np.float64)
    b = oracle.sync(rod.u0, np.float32(rod.r), rod.c1, rod.cN, rod.K)
    assert np.abs(a - b).max() <= 4 * rod.K * np.finfo(np.float32).eps * 2.0
    assert np.abs(a - b).max() > 0  # it really is float arithmetic


def _fp32_inputs(N, seed):
    rng = np.random.default_rng(seed)
    # float32 values over several binades, so that the roundings of every
    # operation land in different places
    u0 = (rng.uniform(-1, 1, size=N) * 2.0 ** rng.integers(-6, 7, size=N)).astype(np.float32)
    return u0, np.float32(0.37), np.float32(0.3125), np.float32(-1.7)


def test_sync_fp32_mode_rounds_each_operation_once():
    """The FP32 mode against an exact-rational restatement of the FP32 order
    of Section 4's kernels (uR - 2u, + uL, fused r*s + u, each rounded to the
    nearest binary32 once), bit for bit."""
    u0, r, c1, cN = _fp32_inputs(24, 7)
    got = oracle.sync(u0, r, c1, cN, 14, dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), pins.fp32_sync_exact(u0, r, c1, cN, 14).view(np.uint32))


def test_sync_fp64_rounds_each_operation_once():
    """The FP64 sweep on general (non-dyadic) data against the same
    exact-rational restatement with binary64 roundings, bit for bit."""
    rng = np.random.default_rng(8)
    u0 = rng.uniform(-1, 1, size=24) * 2.0 ** rng.integers(-30, 31, size=24)
    got = oracle.sync(u0, 0.3712, 0.1, -2.5, 14)
    assert np.array_equal(got.view(np.uint64), pins.fp64_sync_exact(u0, 0.3712, 0.1, -2.5, 14).view(np.uint64))


@pytest.mark.parametrize("S,q,seed", [(4, 3, 1), (24, 2, 2), (3, 4, 3)])
def test_async_fp32_mode_rounds_each_operation_once(S, q, seed):
    """The FP32 switched system (Eq. eqn:async) against the same exact
    roundings with delayed reads from the kept history, bit for bit."""
    u0, r, c1, cN = _fp32_inputs(24, 10 + seed)
    K = 12
    tr = inputs.delay_trace(K, S, q, seed=seed)
    got = oracle.async_replay(u0, r, c1, cN, S, q, K, tr, dtype=np.float32)
    want = pins.fp32_async_exact(u0, r, c1, cN, S, q, tr)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# --------------------------------------------------------------------------- async


def test_async_zero_trace_equals_sync_bitwise():
    """All delays 0 (k* = k) reduces Eq. (eqn:async) to Eq. (eqn:sync)."""
    rod = inputs.small_rod(K=1000)
    tr = np.zeros((rod.K, 7, 2), dtype=np.uint8)
    a = oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, rod.K, tr)
    b = oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K)
    assert np.array_equal(a, b)
    a32 = oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, rod.K, tr, dtype=np.float32)
    b32 = oracle.sync(rod.u0, rod.r, rod.c1, rod.cN, rod.K, dtype=np.float32)
    assert np.array_equal(a32, b32)


@pytest.mark.parametrize("N,S,q,K,seed", [(6, 2, 2, 14, 0), (9, 3, 3, 16, 1), (12, 4, 3, 12, 2),
                                          (7, 7, 2, 14, 3), (10, 5, 1, 16, 4), (11, 2, 4, 10, 5)])
def test_async_brute_force_switched_system_exact(N, S, q, K, seed):
    """Exact rational switched system on the augmented state, one explicit
    block matrix per step, against the oracle bit for bit (dyadic data,
    r = 1/4)."""
    rng = np.random.default_rng(seed)
    u0 = rng.integers(-16, 17, size=N) / 16.0
    tr = rng.integers(0, q, size=(K, S - 1, 2)).astype(np.uint8)
    # clamp as the model requires (no state before k = 0) for the brute force
    trc = np.minimum(tr, np.arange(K)[:, None, None]).astype(np.uint8)
    exact = pins.brute_async_fraction(u0, Fraction(1, 4), 0.25, -0.75, S, q, trc)
    got = oracle.async_replay(u0, 0.25, 0.25, -0.75, S, q, K, tr)
    assert [Fraction(v) for v in got] == exact


def test_async_sides_are_not_interchangeable():
    """Swapping the two sides of the trace changes the result: the pin above
    would catch a side mix-up."""
    rng = np.random.default_rng(9)
    N, S, q, K = 10, 2, 3, 12
    u0 = rng.integers(-16, 17, size=N) / 16.0
    tr = np.zeros((K, 1, 2), dtype=np.uint8)
    tr[5:, 0, 0] = 2
    a = oracle.async_replay(u0, 0.25, 0.0, 0.0, S, q, K, tr)
    b = oracle.async_replay(u0, 0.25, 0.0, 0.0, S, q, K, tr[:, :, ::-1].copy())
    assert not np.array_equal(a, b)


def test_async_rejects_delay_outside_window():
    rod = inputs.small_rod(K=10)
    tr = np.zeros((10, 7, 2), dtype=np.uint8)
    tr[3, 2, 1] = 3
    with pytest.raises(oracle.OracleError):
        oracle.async_replay(rod.u0, rod.r, rod.c1, rod.cN, 8, 3, 10, tr)


@pytest.mark.parametrize("r", [0.1, 0.5])
def test_async_maximum_principle(r):
    rng = np.random.default_rng(4)
    N, S, q, K = 300, 6, 3, 400
    u0 = rng.uniform(-1, 1, size=N)
    tr = inputs.delay_trace(K, S, q, seed=7)
    u = oracle.async_replay(u0, r, 0.2, -0.3, S, q, K, tr)
    lo, hi = min(u0[1:-1].min(), 0.2, -0.3), max(u0[1:-1].max(), 0.2, -0.3)
    assert u.min() >= lo - 1e-13 and u.max() <= hi + 1e-13


def test_async_unique_steady_state():
    """Section 5.3: with Dirichlet ends the asynchronous run reaches the same
    unique steady state as the synchronous one, whatever the delays."""
    N, S, q, K = 24, 6, 3, 30000
    u0 = inputs.paper_rod(N=N).u0
    x = inputs.grid_x(N)
    for seed in (0, 1):
        tr = inputs.delay_trace(K, S, q, seed=seed)
        u = oracle.async_replay(u0, 0.5, 1.0, 0.0, S, q, K, tr)
        assert np.abs(u - (1.0 - x)).max() < 1e-12


def test_delay_trace_generator_is_uniform_and_counter_based():
    tr = inputs.delay_trace(2000, 8, 3, seed=0)
    assert tr.shape == (2000, 7, 2) and tr.dtype == np.uint8
    counts = np.bincount(tr.reshape(-1), minlength=3)
    assert counts.size == 3 and np.all(np.abs(counts / tr.size - 1 / 3) < 0.01)
    # counter-based: the first rows do not depend on K
    assert np.array_equal(inputs.delay_trace(50, 8, 3, seed=0), tr[:50])
    # SplitMix64 reference output for seed 0 (first output of the stream)
    assert int(inputs.splitmix64(0, np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


# --------------------------------------------------------------------------- adjoint


def _fd_setup(N=40, K=60, S=4, q=3, seed=0):
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-1, 1, size=N)
    u_obs = rng.uniform(-1, 1, size=N)
    tr = inputs.delay_trace(K, S, q, seed=seed)
    return u0, u_obs, tr


@pytest.mark.parametrize("use_trace", [False, True])
def test_adjoint_central_finite_differences(use_trace):
    """Directional central differences (h = 1e-6, FP64) of the forward oracle
    against the adjoint gradients with respect to u(0) and r."""
    N, K, S, q = 40, 60, 4, 3
    u0, u_obs, tr = _fd_setup(N, K, S, q)
    r, c1, cN = 0.3, 0.1, -0.2

    def loss(u, rr):
        if use_trace:
            uk = oracle.async_replay(u, rr, c1, cN, S, q, K, tr)
        else:
            uk = oracle.sync(u, rr, c1, cN, K)
        return 0.5 * float(np.sum((uk - u_obs) ** 2))

    L, g, gr = oracle.adjoint(u0, r, c1, cN, K, u_obs, S, q, tr if use_trace else None)
    assert abs(L - loss(u0, r)) < 1e-13
    h = 1e-6
    v = np.random.default_rng(1).standard_normal(N)
    fd = (loss(u0 + h * v, r) - loss(u0 - h * v, r)) / (2 * h)
    assert abs(fd - g @ v) < 1e-7 * max(1.0, abs(fd))
    fdr = (loss(u0, r + h) - loss(u0, r - h)) / (2 * h)
    assert abs(fdr - gr) < 1e-6 * max(1.0, abs(fdr))
    assert g[0] == 0.0 and g[-1] == 0.0


@pytest.mark.parametrize("use_trace", [False, True])
def test_adjoint_matches_transposed_matrices(use_trace):
    """The backward sweep equals the transposed product of the explicit step
    matrices (augmented state for the asynchronous run)."""
    N, K, S, q = 12, 25, 3, 3
    u0, u_obs, tr = _fd_setup(N, K, S, q, seed=3)
    if not use_trace:
        tr = np.zeros_like(tr)
    trc = np.minimum(tr, np.arange(K)[:, None, None]).astype(np.uint8)
    r, c1, cN = 0.35, 0.0, 0.5
    L, g, gr = oracle.adjoint(u0, r, c1, cN, K, u_obs, S, q, tr if use_trace else None)
    Lb, gb, grb = pins.brute_adjoint_float(u0, Fraction(r), c1, cN, S, q, trc, u_obs)
    assert abs(L - Lb) < 1e-13
    assert np.abs(g - gb).max() < 1e-13
    assert abs(gr - grb) < 1e-12


def test_adjoint_sync_is_symmetric_power():
    """Synchronous run: the gradient w.r.t. u(0) is A^K applied to
    (u(K) - u_obs) on the interior (A is symmetric on the interior), i.e. one
    more synchronous run with zero ends."""
    N, K = 50, 200
    rng = np.random.default_rng(8)
    u0, u_obs = rng.random(N), rng.random(N)
    r = 0.3
    L, g, _ = oracle.adjoint(u0, r, 0.0, 0.0, K, u_obs)
    uK = pins.closed_form_sync(u0, r, 0.0, 0.0, K)
    lam = uK - u_obs
    lam[0] = lam[-1] = 0.0
    expect = pins.closed_form_sync(lam, r, 0.0, 0.0, K)
    expect[0] = expect[-1] = 0.0
    assert np.abs(g - expect).max() < 1e-12

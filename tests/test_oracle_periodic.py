"""Pins of the periodic-boundary oracle (Section 5.3): Fourier-mode decay,
conservation of the sum in the synchronous run, exact rational brute force of
the circulant system and of the asynchronous switched system on a ring, and
the paper's observation that asynchrony leaves no unique steady state."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1510_08982_gb300 import inputs
from tests import pins

EPS64 = np.finfo(np.float64).eps


@pytest.mark.parametrize("N,m,r,K", [(64, 1, 0.5, 300), (100, 7, 0.25, 1000), (257, 30, 0.45, 500)])
def test_periodic_fourier_mode_decay(N, m, r, K):
    i = np.arange(N)
    lam = 1.0 - 4.0 * r * math.sin(math.pi * m / N) ** 2
    for f in (np.cos, np.sin):
        u0 = f(2 * math.pi * m * i / N)
        got = oracle.sync_periodic(u0, r, K)
        assert np.abs(got - lam ** K * u0).max() <= 4 * K * EPS64 + 1e-15


@pytest.mark.parametrize("N,r,K", [(5, Fraction(1, 4), 20), (16, Fraction(1, 2), 20), (33, Fraction(3, 8), 12)])
def test_periodic_brute_force_exact(N, r, K):
    u0 = np.random.default_rng(N).integers(-16, 17, size=N) / 16.0
    exact = pins.brute_sync_periodic_fraction(u0, r, K)
    assert [Fraction(v) for v in oracle.sync_periodic(u0, float(r), K)] == exact


def test_periodic_sync_conserves_the_sum():
    u0 = np.random.default_rng(0).integers(-64, 65, size=40) / 64.0
    got = oracle.sync_periodic(u0, 0.25, 20)  # dyadic: exact
    assert Fraction(float(got.sum())) == Fraction(float(u0.sum()))
    rod = inputs.paper_rod(N=100)
    got = oracle.sync_periodic(rod.u0, 0.45, 50000)
    assert abs(got.mean() - rod.u0.mean()) < 1e-12
    assert np.abs(got - rod.u0.mean()).max() < 1e-10  # unique steady state: the mean


def test_periodic_half_r_keeps_the_alternating_mode():
    """At r = 1/2 and even N the alternating mode (-1)^i has lambda = -1: the
    synchronous periodic run of the paper's N = 100, r = 0.5 case keeps a
    checkerboard of the initial projection's size, flipping sign each step."""
    rod = inputs.paper_rod(N=100)
    alt = (-1.0) ** np.arange(100)
    c = float(rod.u0 @ alt) / 100
    for K in (20000, 20001):
        got = oracle.sync_periodic(rod.u0, 0.5, K)
        assert np.abs(got - (rod.u0.mean() + c * (-1) ** K * alt)).max() < 1e-10


@pytest.mark.parametrize("N,S,q,K,seed", [(6, 2, 2, 14, 0), (9, 3, 3, 12, 1), (10, 5, 2, 14, 2), (7, 7, 3, 10, 3)])
def test_async_periodic_brute_force_exact(N, S, q, K, seed):
    rng = np.random.default_rng(seed)
    u0 = rng.integers(-16, 17, size=N) / 16.0
    tr = rng.integers(0, q, size=(K, S, 2)).astype(np.uint8)
    trc = np.minimum(tr, np.arange(K)[:, None, None]).astype(np.uint8)
    exact = pins.brute_async_periodic_fraction(u0, Fraction(1, 4), S, q, trc)
    assert [Fraction(v) for v in oracle.async_periodic(u0, 0.25, S, q, K, tr)] == exact


def test_async_periodic_zero_trace_is_sync():
    rod = inputs.paper_rod(N=100)
    tr = np.zeros((500, 4, 2), dtype=np.uint8)
    assert np.array_equal(oracle.async_periodic(rod.u0, 0.5, 4, 3, 500, tr), oracle.sync_periodic(rod.u0, 0.5, 500))


def test_async_periodic_has_no_unique_steady_state():
    """Section 5.3 / Fig. 6: asynchronous periodic runs from the same u(0)
    flatten to constants that depend on the delays (the sum is not
    conserved), unlike the synchronous run."""
    rod = inputs.paper_rod(N=100)
    K, S, q = 60000, 10, 3
    finals = []
    for seed in (0, 1):
        u = oracle.async_periodic(rod.u0, 0.5, S, q, K, inputs.periodic_delay_trace(K, S, q, seed=seed))
        assert u.max() - u.min() < 1e-9          # it does converge to a constant ...
        finals.append(u.mean())
    assert abs(finals[0] - finals[1]) > 1e-6      # ... but not to a unique one
    assert abs(finals[0] - rod.u0.mean()) > 1e-6


@pytest.mark.parametrize("S,q,seed", [(1, 1, 0), (2, 3, 1), (5, 2, 2), (20, 3, 3)])
def test_periodic_fp32_mode_rounds_each_operation_once(S, q, seed):
    """The FP32 ring, synchronous (S = 1) and driven by ring traces, against the
    exact-rational restatement of the FP32 operation order with each operation
    rounded once to the nearest binary32, bit for bit."""
    rng = np.random.default_rng(40 + seed)
    N, K = 20, 12
    u0 = (rng.uniform(-1, 1, size=N) * 2.0 ** rng.integers(-5, 6, size=N)).astype(np.float32)
    r = np.float32(0.4375)
    if S == 1:
        got = oracle.sync_periodic(u0, r, K, dtype=np.float32)
        want = pins.fp32_periodic_exact(u0, r, K)
    else:
        tr = inputs.periodic_delay_trace(K, S, q, seed=seed)
        got = oracle.async_periodic(u0, r, S, q, K, tr, dtype=np.float32)
        want = pins.fp32_periodic_exact(u0, r, K, S, q, tr)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))

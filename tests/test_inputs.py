"""The seeded input generators against the workload recipes they implement:
sizes, ranges, closed-form initial states, the spectral content of the
sine-mode states, and SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) against
a scalar restatement of its published definition."""
from __future__ import annotations

import math

import numpy as np
from scipy.fft import dst

from paper_1510_08982_gb300 import inputs

MASK = (1 << 64) - 1


def splitmix64_scalar(seed, j):
    """The j-th output of SplitMix64: state advanced j+1 times by the golden
    gamma, then the two xor-shift-multiply rounds and a final xor-shift."""
    z = (seed + (j + 1) * 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_splitmix64_matches_scalar_definition():
    j = np.arange(1000, dtype=np.uint64)
    for seed in (0, 1, 1234567, (1 << 63) + 5, MASK):
        got = inputs.splitmix64(seed, j)
        assert [int(x) for x in got] == [splitmix64_scalar(seed, int(k)) for k in range(1000)]


def test_delay_traces_index_the_generator():
    K, S, q, seed = 37, 6, 3, 9
    tr = inputs.delay_trace(K, S, q, seed)
    assert tr.shape == (K, S - 1, 2) and tr.dtype == np.uint8 and tr.max() < q
    for k, b, s in [(0, 0, 0), (5, 3, 1), (36, 4, 1)]:
        assert tr[k, b, s] == splitmix64_scalar(seed, (k * (S - 1) + b) * 2 + s) % q
    pt = inputs.periodic_delay_trace(K, S, q, seed)
    assert pt.shape == (K, S, 2) and pt.max() < q
    assert pt[7, 5, 1] == splitmix64_scalar(seed, (7 * S + 5) * 2 + 1) % q
    assert inputs.delay_trace(10, 1, 3).shape == (10, 0, 2)


def test_small_rod_recipe():
    rod = inputs.small_rod()
    x = np.arange(1024) / 1023.0
    assert (rod.N, rod.K, rod.r, rod.c1, rod.cN) == (1024, 10_000, 0.4, 0.0, 1.0)
    assert np.allclose(rod.u0, np.sin(math.pi * x) + 0.5 * np.sin(7 * math.pi * x) + x, atol=1e-15)


def test_sine_mode_rod_has_at_most_16_modes_below_513():
    rod = inputs.sine_mode_rod(K=10)
    assert (rod.N, rod.r, rod.c1, rod.cN) == (1 << 20, 0.25, -1.0, 1.0)
    # DST-I of the interior: mode m of sin(m pi x_i) has coefficient a_m (N - 1)
    a = dst(rod.u0[1:-1], type=1) / (rod.N - 1)
    active = np.nonzero(np.abs(a) > 1e-9)[0] + 1
    assert 1 <= active.size <= 16 and active.max() <= 512
    assert np.allclose(rod.u0, inputs.sine_mode_rod(K=10).u0)  # seeded


def test_paper_rod_recipe():
    rod = inputs.paper_rod()
    assert (rod.N, rod.r, rod.c1, rod.cN) == (100, 0.5, 1.0, 0.0)
    i = np.arange(100)
    assert np.allclose(rod.u0, np.cos(3 * math.pi * i / 198.0) ** 2, atol=1e-15)
    assert abs(rod.u0[0] - 1.0) < 1e-15


def test_uneven_rods_ranges():
    rods = inputs.uneven_rods()
    N = np.array([r.N for r in rods])
    K = np.array([r.K for r in rods])
    r = np.array([r_.r for r_ in rods])
    assert len(rods) == 4096
    assert N.min() >= 256 and N.max() <= 65536 and K.min() >= 1000 and K.max() <= 100_000
    assert r.min() >= 0.05 and r.max() <= 0.5
    assert all(-1 <= x.c1 <= 1 and -1 <= x.cN <= 1 for x in rods)
    # log-uniform: the median is near the geometric mean of the range
    assert abs(math.log2(np.median(N)) - 12) < 0.2 and abs(math.log10(np.median(K)) - 4) < 0.1


def test_inverse_problem_rods_and_noise():
    rods = inputs.inverse_problem_rods(n_rods=8, N=4096, K=5)
    assert all(0.1 <= x.r <= 0.45 and x.c1 == 0.0 and x.cN == 0.0 and x.N == 4096 for x in rods)
    for x in rods:
        a = dst(x.u0[1:-1], type=1) / (x.N - 1)
        active = np.nonzero(np.abs(a) > 1e-9)[0] + 1
        assert active.size <= 8 and active.max() <= 64
    e = inputs.observation_noise(200_000, seed=1)
    assert abs(e.std() - 1e-2) < 1e-4 and abs(e.mean()) < 1e-4

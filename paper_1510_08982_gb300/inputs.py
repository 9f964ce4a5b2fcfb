"""Seeded synthetic inputs for the 1D heat-equation runs.

This module holds no arithmetic of the method itself (no stencil, no delay
model): it only draws initial conditions, rod descriptors and delay sequences
from fixed seeds, so that the CUDA library and the CPU oracle are fed the same
numbers.  It imports neither of them.

Grid convention: N points, 0-based storage, x_i = i/(N-1), i = 0..N-1 (the
paper's x_i = (i-1)/(N-1) on 1-based i).  The Dirichlet end values c1 and cN
are forced onto u[0] and u[N-1] by both implementations, so the generators do
not set them.

Delay sequences use SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) as a counter-based generator:
the delay of step k, boundary b and side s is the j-th output of the SplitMix64
stream seeded with ``seed``, j = (k*(S-1) + b)*2 + s, reduced mod q:

    z = seed + (j + 1) * 0x9E3779B97F4A7C15          (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    d = (z ^ (z >> 31)) mod q
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def grid_x(N: int) -> np.ndarray:
    """x_i = i/(N-1), i = 0..N-1, in float64."""
    return np.arange(N, dtype=np.float64) / float(N - 1)


def splitmix64(seed: int, j: np.ndarray) -> np.ndarray:
    """The j-th outputs (j >= 0, uint64 array) of SplitMix64 seeded with ``seed``."""
    j = np.asarray(j, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (j + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def delay_trace(K: int, S: int, q: int, seed: int = 0) -> np.ndarray:
    """Delays i.i.d. uniform in {0, ..., q-1}, shape (K, S-1, 2), uint8."""
    if S < 2:
        return np.zeros((K, 0, 2), dtype=np.uint8)
    j = np.arange(K * (S - 1) * 2, dtype=np.uint64)
    d = splitmix64(seed, j) % np.uint64(q)
    return d.astype(np.uint8).reshape(K, S - 1, 2)


def periodic_delay_trace(K: int, S: int, q: int, seed: int = 0) -> np.ndarray:
    """Delays for the periodic ring of S segments (S boundaries): shape
    (K, S, 2), the j-th SplitMix64 output with j = (k*S + b)*2 + s, mod q."""
    j = np.arange(K * S * 2, dtype=np.uint64)
    d = splitmix64(seed, j) % np.uint64(q)
    return d.astype(np.uint8).reshape(K, S, 2)


def sine_sum(N: int, modes, amps) -> np.ndarray:
    """sum_j amps[j] * sin(modes[j] * pi * x_i), float64."""
    x = grid_x(N)
    u = np.zeros(N, dtype=np.float64)
    for m, a in zip(modes, amps):
        u += float(a) * np.sin(float(m) * math.pi * x)
    return u


# ---------------------------------------------------------------- workloads


@dataclass
class Rod:
    """One rod: N points, K steps, coefficient r, Dirichlet ends c1, cN and u(0)."""
    N: int
    K: int
    r: float
    c1: float
    cN: float
    u0: np.ndarray


def small_rod(N: int = 1024, K: int = 10_000) -> Rod:
    """Plain method, small: N=1024, r=0.4, K=1e4, c1=0, cN=1,
    u(0) = sin(pi x) + 0.5 sin(7 pi x) + x."""
    x = grid_x(N)
    u0 = np.sin(math.pi * x) + 0.5 * np.sin(7 * math.pi * x) + x
    return Rod(N=N, K=K, r=0.4, c1=0.0, cN=1.0, u0=u0)


def sine_mode_rod(N: int = 1 << 20, K: int = 100_000, seed: int = 0, n_modes: int = 16, m_max: int = 512,
                  r: float = 0.25, c1: float = -1.0, cN: float = 1.0) -> Rod:
    """Sync vs async at scale: N=2^20, r=0.25, K=1e5, c1=-1, cN=1, u(0) a sum of
    16 sine modes, m uniform in [1, 512], amplitudes N(0,1), from ``seed``."""
    rng = np.random.default_rng(seed)
    m = rng.integers(1, min(m_max, N - 2) + 1, size=n_modes)
    a = rng.standard_normal(n_modes)
    return Rod(N=N, K=K, r=r, c1=c1, cN=cN, u0=sine_sum(N, m, a))


def uniform_rod(N: int = 1 << 26, K: int = 10_000, r: float = 0.25, seed: int = 0) -> Rod:
    """Bandwidth sweep: c1 = cN = 0, u(0) i.i.d. uniform [0, 1) from ``seed``."""
    rng = np.random.default_rng(seed)
    return Rod(N=N, K=K, r=r, c1=0.0, cN=0.0, u0=rng.random(N))


def paper_rod(N: int = 100, K: int = 1000) -> Rod:
    """The paper's own run (Section 5): r = 0.5, u_i = cos^2(3 pi i / (2(N-1)))
    on 0-based i, ends 1 and 0.  The paper does not give the step count; 1000 is
    a choice."""
    i = np.arange(N, dtype=np.float64)
    u0 = np.cos(3.0 * math.pi * i / (2.0 * (N - 1))) ** 2
    return Rod(N=N, K=K, r=0.5, c1=1.0, cN=0.0, u0=u0)


def uneven_rods(n_rods: int = 4096, seed: int = 0, N_lo: int = 256, N_hi: int = 65536, K_lo: int = 1000,
                K_hi: int = 100_000, r_lo: float = 0.05, r_hi: float = 0.5, n_modes: int = 8,
                m_cap: int = 64) -> list[Rod]:
    """Batched uneven rods: N log-uniform in [N_lo, N_hi], K log-uniform in
    [K_lo, K_hi], r uniform in [r_lo, r_hi], c1 and cN uniform in [-1, 1],
    u(0) a sum of 8 sine modes (m uniform in [1, min(64, N-2)], amplitudes
    N(0,1)), all from one seed."""
    rng = np.random.default_rng(seed)
    Ns = np.exp(rng.uniform(math.log(N_lo), math.log(N_hi), size=n_rods)).astype(np.int64)
    Ns = np.clip(Ns, N_lo, N_hi)
    Ks = np.exp(rng.uniform(math.log(K_lo), math.log(K_hi), size=n_rods)).astype(np.int64)
    Ks = np.clip(Ks, K_lo, K_hi)
    rs = rng.uniform(r_lo, r_hi, size=n_rods)
    c1s = rng.uniform(-1.0, 1.0, size=n_rods)
    cNs = rng.uniform(-1.0, 1.0, size=n_rods)
    rods = []
    for j in range(n_rods):
        N = int(Ns[j])
        m = rng.integers(1, min(m_cap, N - 2) + 1, size=n_modes)
        a = rng.standard_normal(n_modes)
        rods.append(Rod(N=N, K=int(Ks[j]), r=float(rs[j]), c1=float(c1s[j]), cN=float(cNs[j]),
                        u0=sine_sum(N, m, a)))
    return rods


def inverse_problem_rods(n_rods: int = 256, N: int = 65536, K: int = 20_000, seed: int = 0, n_modes: int = 8,
                         m_cap: int = 64) -> list[Rod]:
    """Adjoint / inverse problem: r_true uniform in [0.1, 0.45], smooth u(0)
    (8 sine modes), c1 = cN = 0."""
    rng = np.random.default_rng(seed)
    rods = []
    for _ in range(n_rods):
        m = rng.integers(1, min(m_cap, N - 2) + 1, size=n_modes)
        a = rng.standard_normal(n_modes)
        r = float(rng.uniform(0.1, 0.45))
        rods.append(Rod(N=N, K=K, r=r, c1=0.0, cN=0.0, u0=sine_sum(N, m, a)))
    return rods


def observation_noise(n: int, seed: int, sigma: float = 1e-2) -> np.ndarray:
    """Gaussian noise of variance sigma^2 (1e-4 by default) for u_obs."""
    return np.random.default_rng(seed).normal(0.0, sigma, size=n)

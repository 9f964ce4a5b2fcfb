"""Independent checks of the oracle: closed forms and brute force.

Nothing here calls the oracle or the CUDA library.  Each helper restates what
the mathematics fixes for the update of Section 2 (Eq. eqn:sync) and Section 3
(Eq. eqn:async) in a form different from the oracle's sweep:

* closed_form_sync: the discrete sine modes are eigenvectors of the FTCS
  operator with Dirichlet ends; mode m decays by
  lambda_m = 1 - 4 r sin^2(m pi dx / 2) per step, dx = 1/(N-1), and the linear
  profile between c1 and cN is a fixed point.
* brute_sync_fraction: the N x N matrix A of Eq. (eqn:sync), applied K times in
  exact rational arithmetic.
* brute_async_fraction: the switched system on the augmented state
  z(k) = [u(k); u(k-1); ...; u(k-q+1)] with one explicit block matrix per step
  built from the delays; times before 0 are served by z(0) = [u0; ...; u0].
* brute_adjoint: gradients by the transposed products of those matrices.
* fp64_sync_exact, fp32_sync_exact, fp32_async_exact, fp32_periodic_exact:
  the operation order of Section 4's kernels with every operation's exact
  rational result rounded once to the nearest binary64 or binary32 (ties to
  even), so that the oracle is checked bit for bit on general data rather than
  within a bound.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
from scipy.fft import dst, idst


def forced(u0, c1, cN):
    u = np.array(u0, dtype=np.float64, copy=True)
    u[0] = c1
    u[-1] = cN
    return u


def closed_form_sync(u0, r, c1, cN, K):
    """u(K) from the sine-mode expansion of u(0) - u_ss on the interior."""
    u0 = forced(u0, c1, cN)
    N = u0.size
    n = N - 2
    x = np.arange(N, dtype=np.float64) / (N - 1)
    uss = c1 + (cN - c1) * x
    f = (u0 - uss)[1:-1]
    F = dst(f, type=1)
    m = np.arange(1, n + 1, dtype=np.float64)
    lam = 1.0 - 4.0 * r * np.sin(m * math.pi / (2.0 * (N - 1))) ** 2
    # lam^K: lam may be negative for r > 1/4 and high modes
    lamK = np.sign(lam) ** (K % 2) * np.exp(K * np.log(np.abs(lam))) if K > 0 else np.ones_like(lam)
    out = uss.copy()
    out[1:-1] += idst(F * lamK, type=1)
    return out


def _frac(v):
    return Fraction(v) if not isinstance(v, Fraction) else v


def sync_matrix_fraction(N, r):
    r = _frac(r)
    A = [[Fraction(0)] * N for _ in range(N)]
    A[0][0] = Fraction(1)
    A[N - 1][N - 1] = Fraction(1)
    for i in range(1, N - 1):
        A[i][i - 1] = r
        A[i][i] = 1 - 2 * r
        A[i][i + 1] = r
    return A


def matvec(A, x):
    return [sum((a * b for a, b in zip(row, x) if a != 0), Fraction(0)) for row in A]


def brute_sync_fraction(u0, r, c1, cN, K):
    """A^K u(0), exact, with the ends forced first."""
    u = [_frac(v) for v in u0]
    u[0] = _frac(c1)
    u[-1] = _frac(cN)
    A = sync_matrix_fraction(len(u), r)
    for _ in range(K):
        u = matvec(A, u)
    return u


def segment_of(N, S, offsets=None):
    """Segment index of every point: the standard split (the first N mod S
    segments one point longer), or the split given by S+1 offsets."""
    if offsets is not None:
        seg = []
        for s in range(len(offsets) - 1):
            seg += [s] * (int(offsets[s + 1]) - int(offsets[s]))
        return seg
    base, extra = divmod(N, S)
    seg, s, count = [], 0, 0
    for s in range(S):
        seg += [s] * (base + (1 if s < extra else 0))
    return seg


def async_step_matrix(N, r, S, q, dk, offsets=None):
    """Block matrix (qN x qN) for one step of Eq. (eqn:async).

    dk has shape (S-1, 2): dk[b][0] is the delay of segment b's read of its
    right neighbour, dk[b][1] that of segment b+1's read of its left
    neighbour.  Block j of z holds u(k-j).  Delays must already be clamped to
    at most q-1 (the augmented state has q blocks)."""
    r = _frac(r)
    seg = segment_of(N, S, offsets)
    M = [[Fraction(0)] * (q * N) for _ in range(q * N)]
    M[0][0] = Fraction(1)
    M[N - 1][N - 1] = Fraction(1)
    for i in range(1, N - 1):
        jl = int(dk[seg[i - 1]][1]) if seg[i - 1] != seg[i] else 0
        jr = int(dk[seg[i]][0]) if seg[i + 1] != seg[i] else 0
        M[i][i] += 1 - 2 * r
        M[i][jl * N + i - 1] += r
        M[i][jr * N + i + 1] += r
    for j in range(1, q):  # shift the history down by one block
        for i in range(N):
            M[j * N + i][(j - 1) * N + i] = Fraction(1)
    return M


def brute_async_fraction(u0, r, c1, cN, S, q, trace, offsets=None):
    """Exact u(K) of the switched system driven by trace (K, S-1, 2); the
    segments are the standard split or the one given by offsets."""
    N = len(u0)
    u = [_frac(v) for v in u0]
    u[0] = _frac(c1)
    u[-1] = _frac(cN)
    z = u * q
    trace = np.asarray(trace)
    for k in range(trace.shape[0]):
        M = async_step_matrix(N, r, S, q, trace[k], offsets)
        z = matvec(M, z)
    return z[:N]


def brute_adjoint_float(u0, r, c1, cN, S, q, trace, u_obs):
    """Loss and gradient w.r.t. u(0) through the transposed step matrices
    (float64 products of the exact matrices).  Also returns dL/dr by the exact
    derivative of each step matrix with respect to r."""
    N = len(u0)
    trace = np.asarray(trace)
    K = trace.shape[0]
    mats, dmats = [], []
    for k in range(K):
        M = np.array(async_step_matrix(N, r, S, q, trace[k]), dtype=np.float64)
        mats.append(M)
        # d M / d r: the r-dependent entries are +1 (neighbour reads) and -2 (self)
        Mp = np.array(async_step_matrix(N, Fraction(1), S, q, trace[k]), dtype=np.float64)
        M0 = np.array(async_step_matrix(N, Fraction(0), S, q, trace[k]), dtype=np.float64)
        dmats.append(Mp - M0)
    u = forced(u0, c1, cN)
    zs = [np.tile(u, q)]
    for M in mats:
        zs.append(M @ zs[-1])
    uK = zs[-1][:N]
    e = uK - np.asarray(u_obs, dtype=np.float64)
    loss = 0.5 * float(np.sum(e * e))
    lam = np.zeros(q * N)
    lam[1:N - 1] = e[1:N - 1]
    gr = 0.0
    for k in range(K - 1, -1, -1):
        gr += float(lam @ (dmats[k] @ zs[k]))
        lam = mats[k].T @ lam
    g = lam.reshape(q, N).sum(axis=0)  # z(0) repeats u(0) in every block
    g[0] = 0.0
    g[-1] = 0.0
    return loss, g, gr


# ----------------------------------------------------------------------------- periodic boundary


def periodic_matrix_fraction(N, r):
    """Circulant matrix of the periodic update (Section 5.3)."""
    r = _frac(r)
    A = [[Fraction(0)] * N for _ in range(N)]
    for i in range(N):
        A[i][i] += 1 - 2 * r
        A[i][(i - 1) % N] += r
        A[i][(i + 1) % N] += r
    return A


def brute_sync_periodic_fraction(u0, r, K):
    u = [_frac(v) for v in u0]
    A = periodic_matrix_fraction(len(u), r)
    for _ in range(K):
        u = matvec(A, u)
    return u


def async_periodic_step_matrix(N, r, S, q, dk):
    """Block matrix for one periodic asynchronous step; dk has shape (S, 2):
    boundary b joins segment b and (b+1) mod S."""
    r = _frac(r)
    seg = segment_of(N, S)
    M = [[Fraction(0)] * (q * N) for _ in range(q * N)]
    for i in range(N):
        il, ir = (i - 1) % N, (i + 1) % N
        jl = int(dk[seg[il]][1]) if seg[il] != seg[i] else 0
        jr = int(dk[seg[i]][0]) if seg[ir] != seg[i] else 0
        M[i][i] += 1 - 2 * r
        M[i][jl * N + il] += r
        M[i][jr * N + ir] += r
    for j in range(1, q):
        for i in range(N):
            M[j * N + i][(j - 1) * N + i] = Fraction(1)
    return M


def brute_async_periodic_fraction(u0, r, S, q, trace):
    N = len(u0)
    z = [_frac(v) for v in u0] * q
    trace = np.asarray(trace)
    for k in range(trace.shape[0]):
        z = matvec(async_periodic_step_matrix(N, r, S, q, trace[k]), z)
    return z[:N]


# ----------------------------------------------------------------------------- asynchronous, temporally blocked


def brute_async_blocked_fraction(u0, r, c1, cN, S, q, T, K, trace, offsets=None):
    """Exact state after K steps of the blocked asynchronous run, written as
    matrix powers on whole vectors: for block b and segment s the composite
    vector z = W_b, with the T points left of the segment taken from W_{b-dL}
    and the T points right of it from W_{b-dR}, is multiplied by the
    synchronous matrix tb times; the segment's own entries of the product are
    its part of W_{b+1}.  A's rows for the segment's own points reach at most
    tb <= T points out, so the whole-vector product needs no tile edges.
    trace: (ceil(K/T), S-1, 2), delays already clamped to b."""
    N = len(u0)
    u = [_frac(v) for v in u0]
    u[0] = _frac(c1)
    u[-1] = _frac(cN)
    A = sync_matrix_fraction(N, r)
    if offsets is not None:
        off = [int(x) for x in offsets]
    else:
        off = [0]
        base, extra = divmod(N, S)
        for s in range(S):
            off.append(off[-1] + base + (1 if s < extra else 0))
    W = [u]
    trace = np.asarray(trace)
    nb = (K + T - 1) // T
    for b in range(nb):
        tb = min(T, K - b * T)
        new = list(W[b])
        for s in range(S):
            lo, hi = off[s], off[s + 1]
            z = list(W[b])
            if s > 0:
                bl = b - int(trace[b][s - 1][1])
                for i in range(max(lo - T, 0), lo):
                    z[i] = W[bl][i]
            if s + 1 < S:
                br = b - int(trace[b][s][0])
                for i in range(hi, min(hi + T, N)):
                    z[i] = W[br][i]
            for _ in range(tb):
                z = matvec(A, z)
            new[lo:hi] = z[lo:hi]
        W.append(new)
    return W[nb]


def brute_async_blocked_periodic_fraction(u0, r, S, q, T, K, trace):
    """The blocked asynchronous model on the periodic ring, exactly: for block
    b and segment s the composite vector (W_b with the T points before the
    segment, indices mod N, from W_{b-dL} and the T points after it from
    W_{b-dR}) is multiplied tb times by the circulant matrix; the segment's
    entries of the product are its part of W_{b+1}.  trace: (nb, S, 2),
    delays clamped to b; boundary b joins segment b and (b+1) mod S."""
    N = len(u0)
    A = periodic_matrix_fraction(N, r)
    off = [0]
    base, extra = divmod(N, S)
    for s in range(S):
        off.append(off[-1] + base + (1 if s < extra else 0))
    W = [[_frac(v) for v in u0]]
    trace = np.asarray(trace)
    nb = (K + T - 1) // T
    for b in range(nb):
        tb = min(T, K - b * T)
        new = list(W[b])
        for s in range(S):
            lo, hi = off[s], off[s + 1]
            bl = b - int(trace[b][(s - 1) % S][1])
            br = b - int(trace[b][s][0])
            z = list(W[b])
            for x in range(1, T + 1):
                z[(lo - x) % N] = W[bl][(lo - x) % N]
                z[(hi - 1 + x) % N] = W[br][(hi - 1 + x) % N]
            for _ in range(tb):
                z = matvec(A, z)
            new[lo:hi] = z[lo:hi]
        W.append(new)
    return W[nb]


# ----------------------------------------------------------------------------- FP32 operation order


def round_to_float32(q):
    """The binary32 value nearest to the rational q, ties to even (IEEE 754
    round to nearest), returned as a Python float (exact: binary32 values are
    binary64 values).  |q| must be below 2^128."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()  # 2^e <= a < 2^(e+1) after the fix-ups
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)  # subnormals share the spacing of the smallest normal binade
    ulp = Fraction(2) ** (e - 23)
    n, rem = divmod(a, ulp)
    n = int(n)
    half = ulp / 2
    if rem > half or (rem == half and n % 2 == 1):
        n += 1
    return sign * float(n * ulp)


def round_to_float64(q):
    """The binary64 value nearest to the rational q, ties to even: Python's
    int / int division (which float(Fraction) uses) is correctly rounded."""
    return float(q)


def _update(r, uL, u, uR, rnd):
    """One interior update in the order of the paper's kernels (Section 4):
    t = uR - 2u rounded (2u is exact), s = t + uL rounded, then r*s + u with a
    single rounding (the fused multiply-add); rnd rounds a rational."""
    t = Fraction(rnd(uR - 2 * u))
    s = Fraction(rnd(t + uL))
    return Fraction(rnd(r * s + u))


def _fp32_update(r, uL, u, uR):
    return _update(r, uL, u, uR, round_to_float32)


def fp64_sync_exact(u0, r, c1, cN, K):
    """u(K) of Eq. (eqn:sync) in FP64 with every operation's exact rational
    result rounded once to the nearest binary64."""
    u = [Fraction(float(v)) for v in u0]
    u[0], u[-1] = Fraction(float(c1)), Fraction(float(cN))
    R = Fraction(float(r))
    for _ in range(K):
        u = [u[0]] + [_update(R, u[i - 1], u[i], u[i + 1], round_to_float64) for i in range(1, len(u) - 1)] + [u[-1]]
    return np.array([float(x) for x in u])


def fp32_sync_exact(u0, r, c1, cN, K):
    """u(K) of Eq. (eqn:sync) in FP32, every operation rounded exactly once
    from its exact rational value (inputs must be binary32 values)."""
    u = [Fraction(float(v)) for v in u0]
    u[0], u[-1] = Fraction(float(c1)), Fraction(float(cN))
    R = Fraction(float(r))
    for _ in range(K):
        u = [u[0]] + [_fp32_update(R, u[i - 1], u[i], u[i + 1]) for i in range(1, len(u) - 1)] + [u[-1]]
    return np.array([float(x) for x in u], dtype=np.float32)


def fp32_async_exact(u0, r, c1, cN, S, q, trace):
    """u(K) of Eq. (eqn:async) in FP32 with the same exact roundings: a read
    across a segment boundary takes the neighbour's value at step k - d
    (d clamped to k) from the kept history of states."""
    N = len(u0)
    u = [Fraction(float(v)) for v in u0]
    u[0], u[-1] = Fraction(float(c1)), Fraction(float(cN))
    R = Fraction(float(r))
    seg = segment_of(N, S)
    hist = [u]
    trace = np.asarray(trace)
    for k in range(trace.shape[0]):
        cur = hist[-1]
        nxt = [cur[0]] + [Fraction(0)] * (N - 2) + [cur[-1]]
        for i in range(1, N - 1):
            uL, uR = cur[i - 1], cur[i + 1]
            if seg[i - 1] != seg[i]:
                uL = hist[k - min(int(trace[k][seg[i - 1]][1]), k)][i - 1]
            if seg[i + 1] != seg[i]:
                uR = hist[k - min(int(trace[k][seg[i]][0]), k)][i + 1]
            nxt[i] = _fp32_update(R, uL, cur[i], uR)
        hist.append(nxt)
    return np.array([float(x) for x in hist[-1]], dtype=np.float32)


def fp32_periodic_exact(u0, r, K, S=1, q=1, trace=None):
    """u(K) on the periodic ring (Section 5.3) in FP32 with the exact single
    roundings of fp32_sync_exact; with a trace (K, S, 2), a read across
    boundary b (segment b to segment (b+1) mod S) takes the neighbour's value
    at step k - d, d clamped to k."""
    N = len(u0)
    R = Fraction(float(r))
    seg = segment_of(N, S)
    hist = [[Fraction(float(v)) for v in u0]]
    for k in range(K):
        cur = hist[-1]
        nxt = []
        for i in range(N):
            il, ir = (i - 1) % N, (i + 1) % N
            tl = tr_ = k
            if trace is not None and seg[il] != seg[i]:
                tl = k - min(int(trace[k][seg[il]][1]), k)
            if trace is not None and seg[ir] != seg[i]:
                tr_ = k - min(int(trace[k][seg[i]][0]), k)
            nxt.append(_fp32_update(R, hist[tl][il], cur[i], hist[tr_][ir]))
        hist.append(nxt)
    return np.array([float(x) for x in hist[-1]], dtype=np.float32)

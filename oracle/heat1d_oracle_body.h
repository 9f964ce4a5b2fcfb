/*
 * Body of the oracle, written once for a generic REAL and included by
 * heat1d_oracle.c for double (suffix _f64) and for float (suffix _f32).
 * TEST INFRASTRUCTURE ONLY (see heat1d_oracle.c).
 */

/* Synchronous run, Section 2 Eq. (eqn:sync) with Dirichlet ends.
 * Double-buffered Jacobi sweep; every interior point is updated from the
 * previous time level only.  out receives u(K) (N values). */
int SUF(oracle_sync)(int64_t N, REAL r, REAL c1, REAL cN, const REAL* u0, int64_t K, REAL* out) {
  if (N < 3 || K < 0 || !u0 || !out) return ORACLE_EINVAL;
  REAL* a = (REAL*)malloc(sizeof(REAL) * (size_t)N);
  REAL* b = (REAL*)malloc(sizeof(REAL) * (size_t)N);
  if (!a || !b) { free(a); free(b); return ORACLE_ENOMEM; }
  memcpy(a, u0, sizeof(REAL) * (size_t)N);
  a[0] = c1;
  a[N - 1] = cN;
  for (int64_t k = 0; k < K; ++k) {
    for (int64_t i = 1; i < N - 1; ++i) {
      REAL uL = a[i - 1], u = a[i], uR = a[i + 1];
      b[i] = FMA(r, (uR - (REAL)2 * u) + uL, u);
    }
    b[0] = c1;
    b[N - 1] = cN;
    REAL* t = a; a = b; b = t;
  }
  memcpy(out, a, sizeof(REAL) * (size_t)N);
  free(a);
  free(b);
  return ORACLE_OK;
}

/* Asynchronous run, Section 3 Eq. (eqn:async), as the switched linear system
 * on the augmented state z(k) = [u(k); u(k-1); ...; u(k-q+1)].
 *
 * The last q+1 full states are kept in a ring hist[t mod (q+1)].  At step k a
 * read that crosses a segment boundary takes the neighbour at time
 * k - min(d, k), d taken from the trace; every other read takes time k.
 * The new state goes into the slot of time k+1, which held time k-q: a time no
 * read of step k can ask for.  out receives u(K).
 *
 * S = 1 (one segment) has no boundaries, and then trace may be NULL. */
int SUF(oracle_async)(int64_t N, REAL r, REAL c1, REAL cN, int64_t S, int q, const REAL* u0, int64_t K,
                      const uint8_t* trace, REAL* out) {
  if (N < 3 || K < 0 || S < 1 || S > N || q < 1 || q > 255 || !u0 || !out) return ORACLE_EINVAL;
  if (S > 1 && K > 0 && !trace) return ORACLE_EINVAL;
  for (int64_t j = 0; S > 1 && j < K * (S - 1) * 2; ++j)
    if (trace[j] >= q) return ORACLE_ETRACE;
  int64_t Q = (int64_t)q + 1;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  int64_t* seg = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  REAL* hist = (REAL*)malloc(sizeof(REAL) * (size_t)N * (size_t)Q);
  if (!off || !seg || !hist) { free(off); free(seg); free(hist); return ORACLE_ENOMEM; }
  oracle_segments(N, S, off);
  for (int64_t s = 0; s < S; ++s)
    for (int64_t i = off[s]; i < off[s + 1]; ++i) seg[i] = s;
#define H(t, i) hist[(size_t)((t) % Q) * (size_t)N + (size_t)(i)]
  for (int64_t i = 0; i < N; ++i) H(0, i) = u0[i];
  H(0, 0) = c1;
  H(0, N - 1) = cN;
  for (int64_t k = 0; k < K; ++k) {
    for (int64_t i = 1; i < N - 1; ++i) {
      int64_t tL = k, tR = k;
      if (seg[i - 1] != seg[i]) { /* segment seg[i] reads its left neighbour: boundary seg[i-1], side 1 */
        int64_t d = trace[(k * (S - 1) + seg[i - 1]) * 2 + 1];
        tL = k - (d < k ? d : k);
      }
      if (seg[i + 1] != seg[i]) { /* segment seg[i] reads its right neighbour: boundary seg[i], side 0 */
        int64_t d = trace[(k * (S - 1) + seg[i]) * 2 + 0];
        tR = k - (d < k ? d : k);
      }
      REAL uL = H(tL, i - 1), u = H(k, i), uR = H(tR, i + 1);
      H(k + 1, i) = FMA(r, (uR - (REAL)2 * u) + uL, u);
    }
    H(k + 1, 0) = c1;
    H(k + 1, N - 1) = cN;
  }
  for (int64_t i = 0; i < N; ++i) out[i] = H(K, i);
#undef H
  free(off);
  free(seg);
  free(hist);
  return ORACLE_OK;
}

/* Periodic boundary, Section 5.3: the two end points are updated too, each
 * with the other as its outer neighbour (u_1 uses u_N, u_N uses u_1), so
 * every point i uses (i-1) mod N and (i+1) mod N.  Synchronous form. */
int SUF(oracle_sync_periodic)(int64_t N, REAL r, const REAL* u0, int64_t K, REAL* out) {
  if (N < 3 || K < 0 || !u0 || !out) return ORACLE_EINVAL;
  REAL* a = (REAL*)malloc(sizeof(REAL) * (size_t)N);
  REAL* b = (REAL*)malloc(sizeof(REAL) * (size_t)N);
  if (!a || !b) { free(a); free(b); return ORACLE_ENOMEM; }
  memcpy(a, u0, sizeof(REAL) * (size_t)N);
  for (int64_t k = 0; k < K; ++k) {
    for (int64_t i = 0; i < N; ++i) {
      REAL uL = a[(i + N - 1) % N], u = a[i], uR = a[(i + 1) % N];
      b[i] = FMA(r, (uR - (REAL)2 * u) + uL, u);
    }
    REAL* t = a; a = b; b = t;
  }
  memcpy(out, a, sizeof(REAL) * (size_t)N);
  free(a);
  free(b);
  return ORACLE_OK;
}

/* Periodic boundary, asynchronous form (Section 5.3 with Section 3's
 * Eq. (eqn:async)): S >= 2 segments on a ring; boundary b joins segment b and
 * segment (b+1) mod S, so there are S boundaries and the trace is
 * uint8[K][S][2] (side 0: segment b reads its right neighbour, side 1:
 * segment (b+1) mod S reads its left neighbour).  Same history scheme as
 * oracle_async. */
int SUF(oracle_async_periodic)(int64_t N, REAL r, int64_t S, int q, const REAL* u0, int64_t K,
                               const uint8_t* trace, REAL* out) {
  if (N < 3 || K < 0 || S < 2 || S > N || q < 1 || q > 255 || !u0 || !out || (K > 0 && !trace))
    return ORACLE_EINVAL;
  for (int64_t j = 0; j < K * S * 2; ++j)
    if (trace[j] >= q) return ORACLE_ETRACE;
  int64_t Q = (int64_t)q + 1;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  int64_t* seg = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  REAL* hist = (REAL*)malloc(sizeof(REAL) * (size_t)N * (size_t)Q);
  if (!off || !seg || !hist) { free(off); free(seg); free(hist); return ORACLE_ENOMEM; }
  oracle_segments(N, S, off);
  for (int64_t s = 0; s < S; ++s)
    for (int64_t i = off[s]; i < off[s + 1]; ++i) seg[i] = s;
#define H(t, i) hist[(size_t)((t) % Q) * (size_t)N + (size_t)(i)]
  for (int64_t i = 0; i < N; ++i) H(0, i) = u0[i];
  for (int64_t k = 0; k < K; ++k) {
    for (int64_t i = 0; i < N; ++i) {
      int64_t il = (i + N - 1) % N, ir = (i + 1) % N;
      int64_t tL = k, tR = k;
      if (seg[il] != seg[i]) { /* left read crosses boundary seg[il] (side 1) */
        int64_t d = trace[(k * S + seg[il]) * 2 + 1];
        tL = k - (d < k ? d : k);
      }
      if (seg[ir] != seg[i]) { /* right read crosses boundary seg[i] (side 0) */
        int64_t d = trace[(k * S + seg[i]) * 2 + 0];
        tR = k - (d < k ? d : k);
      }
      REAL uL = H(tL, il), u = H(k, i), uR = H(tR, ir);
      H(k + 1, i) = FMA(r, (uR - (REAL)2 * u) + uL, u);
    }
  }
  for (int64_t i = 0; i < N; ++i) out[i] = H(K, i);
#undef H
  free(off);
  free(seg);
  free(hist);
  return ORACLE_OK;
}

/* Asynchronous run with temporal blocking: the bounded-delay model of
 * Section 3 applied to blocks of T steps instead of single steps (the paper's
 * PE exchanges one value per step; here a PE exchanges a strip of T edge
 * values once per T steps).  This is a different switched system from
 * Eq. (eqn:async); it is defined as follows.
 *
 *  - Time is cut into blocks of T steps; block b runs from step bT to step
 *    bT + tb, tb = min(T, K - bT).  W_b denotes the full state at step bT.
 *  - Segment s = [lo, hi) starts block b from a tile covering
 *    [lo - T, hi + T) clipped to [0, N): its own points from W_b, the T points
 *    left of lo from W_{b - dL}, the T points right of hi from W_{b - dR},
 *    where dL = trace[(b(S-1) + s-1)*2 + 1] and dR = trace[(b(S-1) + s)*2 + 0]
 *    (the same sides as Eq. (eqn:async)'s trace), each clamped to b.
 *  - It sweeps the tile tb times with the Section 2 update (the tile's two
 *    outermost points and the Dirichlet ends are held), and its own points
 *    after the last sweep are its part of W_{b+1}.  Own points lie at least
 *    T >= tb points inside the tile, so no held tile edge reaches them.
 *  - A halo must lie within the adjacent segment: every segment other than
 *    the first and the last holds at least T points (the first and the last
 *    may be shorter: a halo reaching past a rod end is clipped there).
 *  - The segments are given by S+1 offsets, off[0] = 0 < off[1] < ... <
 *    off[S] = N (oracle_async_blocked_split), or are the standard split of
 *    oracle_segments (oracle_async_blocked, which also asks every segment to
 *    hold at least T points).
 *
 * With every delay 0 this is the synchronous run; with T = 1 it is
 * Eq. (eqn:async) with the same trace.  The last q+1 block states are kept
 * (block b reads W_{b-q+1} .. W_b and writes W_{b+1} into the slot of
 * W_{b-q}).  trace holds ceil(K/T)*(S-1)*2 entries. */
int SUF(oracle_async_blocked_split)(int64_t N, REAL r, REAL c1, REAL cN, int64_t S, const int64_t* off, int q,
                                    int64_t T, const REAL* u0, int64_t K, const uint8_t* trace, REAL* out) {
  if (N < 3 || K < 0 || S < 1 || S > N || q < 1 || q > 255 || T < 1 || !off || !u0 || !out) return ORACLE_EINVAL;
  if (off[0] != 0 || off[S] != N) return ORACLE_EINVAL;
  for (int64_t s = 0; s < S; ++s) {
    if (off[s + 1] <= off[s]) return ORACLE_EINVAL;
    if (s > 0 && s + 1 < S && off[s + 1] - off[s] < T) return ORACLE_EINVAL;
  }
  int64_t nb = (K + T - 1) / T;
  if (S > 1 && nb > 0 && !trace) return ORACLE_EINVAL;
  for (int64_t j = 0; S > 1 && j < nb * (S - 1) * 2; ++j)
    if (trace[j] >= q) return ORACLE_ETRACE;
  int64_t Q = (int64_t)q + 1;
  REAL* W = (REAL*)malloc(sizeof(REAL) * (size_t)N * (size_t)Q);
  REAL* ta = (REAL*)malloc(sizeof(REAL) * (size_t)N);
  REAL* tb_ = (REAL*)malloc(sizeof(REAL) * (size_t)N);
  if (!W || !ta || !tb_) { free(W); free(ta); free(tb_); return ORACLE_ENOMEM; }
#define WB(b, i) W[(size_t)((b) % Q) * (size_t)N + (size_t)(i)]
  for (int64_t i = 0; i < N; ++i) WB(0, i) = u0[i];
  WB(0, 0) = c1;
  WB(0, N - 1) = cN;
  for (int64_t b = 0; b < nb; ++b) {
    int64_t steps = K - b * T < T ? K - b * T : T;
    for (int64_t s = 0; s < S; ++s) {
      int64_t lo = off[s], hi = off[s + 1];
      int64_t tlo = lo - T > 0 ? lo - T : 0, thi = hi + T < N ? hi + T : N; /* tile [tlo, thi) */
      int64_t bl = b, br = b;
      if (s > 0) {
        int64_t d = trace[(b * (S - 1) + (s - 1)) * 2 + 1];
        bl = b - (d < b ? d : b);
      }
      if (s + 1 < S) {
        int64_t d = trace[(b * (S - 1) + s) * 2 + 0];
        br = b - (d < b ? d : b);
      }
      for (int64_t i = tlo; i < thi; ++i) ta[i] = i < lo ? WB(bl, i) : (i >= hi ? WB(br, i) : WB(b, i));
      REAL* x = ta;
      REAL* y = tb_;
      for (int64_t j = 0; j < steps; ++j) {
        for (int64_t i = tlo; i < thi; ++i) {
          if (i == tlo || i == thi - 1 || i == 0 || i == N - 1) {
            y[i] = x[i]; /* held: a tile edge or a Dirichlet end */
          } else {
            REAL uL = x[i - 1], u = x[i], uR = x[i + 1];
            y[i] = FMA(r, (uR - (REAL)2 * u) + uL, u);
          }
        }
        REAL* t = x; x = y; y = t;
      }
      for (int64_t i = lo; i < hi; ++i) WB(b + 1, i) = x[i];
    }
  }
  for (int64_t i = 0; i < N; ++i) out[i] = WB(nb, i);
#undef WB
  free(W);
  free(ta);
  free(tb_);
  return ORACLE_OK;
}

int SUF(oracle_async_blocked)(int64_t N, REAL r, REAL c1, REAL cN, int64_t S, int q, int64_t T,
                              const REAL* u0, int64_t K, const uint8_t* trace, REAL* out) {
  if (N < 3 || S < 1 || S > N || T < 1) return ORACLE_EINVAL;
  if (S > 1 && T > N / S) return ORACLE_EINVAL; /* N / S is the shortest segment */
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  if (!off) return ORACLE_ENOMEM;
  oracle_segments(N, S, off);
  int rc = SUF(oracle_async_blocked_split)(N, r, c1, cN, S, off, q, T, u0, K, trace, out);
  free(off);
  return rc;
}

/* The blocked asynchronous model on the periodic ring (Section 5.3): as
 * oracle_async_blocked, with S >= 2 segments on a ring.  Segment s takes its
 * left halo (the T points before its first point, indices mod N) from
 * W_{b-dL} and its right halo (the T points after its last one) from
 * W_{b-dR}; boundary b joins segment b and (b+1) mod S, so the trace is
 * uint8[ceil(K/T)][S][2] (side 0: segment b reads its right neighbour; side
 * 1: segment (b+1) mod S reads its left one).  No point is held except the
 * tile's two outermost ones.  T may not exceed the shortest segment.  With
 * S = 2 both halos come from the one neighbour; where 2T exceeds its length
 * they share points, each strip keeping its own copy (the tile holds
 * L + 2T values). */
int SUF(oracle_async_blocked_periodic)(int64_t N, REAL r, int64_t S, int q, int64_t T, const REAL* u0, int64_t K,
                                       const uint8_t* trace, REAL* out) {
  if (N < 3 || K < 0 || S < 2 || S > N || q < 1 || q > 255 || T < 1 || !u0 || !out) return ORACLE_EINVAL;
  int64_t nb = (K + T - 1) / T;
  if (T > N / S) return ORACLE_EINVAL;
  if (nb > 0 && !trace) return ORACLE_EINVAL;
  for (int64_t j = 0; j < nb * S * 2; ++j)
    if (trace[j] >= q) return ORACLE_ETRACE;
  int64_t Q = (int64_t)q + 1;
  int64_t M = N / S + 1 + 2 * T; /* longest tile */
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  REAL* W = (REAL*)malloc(sizeof(REAL) * (size_t)N * (size_t)Q);
  REAL* ta = (REAL*)malloc(sizeof(REAL) * (size_t)M);
  REAL* tb_ = (REAL*)malloc(sizeof(REAL) * (size_t)M);
  if (!off || !W || !ta || !tb_) { free(off); free(W); free(ta); free(tb_); return ORACLE_ENOMEM; }
  oracle_segments(N, S, off);
#define WB(b, i) W[(size_t)((b) % Q) * (size_t)N + (size_t)(i)]
  for (int64_t i = 0; i < N; ++i) WB(0, i) = u0[i];
  for (int64_t b = 0; b < nb; ++b) {
    int64_t steps = K - b * T < T ? K - b * T : T;
    for (int64_t s = 0; s < S; ++s) {
      int64_t lo = off[s], hi = off[s + 1], len = hi - lo + 2 * T; /* tile: T + own + T */
      int64_t dl = trace[(b * S + (s + S - 1) % S) * 2 + 1], dr = trace[(b * S + s) * 2 + 0];
      int64_t bl = b - (dl < b ? dl : b), br = b - (dr < b ? dr : b);
      for (int64_t x = 0; x < len; ++x) {
        int64_t g = ((lo - T + x) % N + N) % N;
        ta[x] = x < T ? WB(bl, g) : (x >= len - T ? WB(br, g) : WB(b, g));
      }
      REAL* xa = ta;
      REAL* ya = tb_;
      for (int64_t j = 0; j < steps; ++j) {
        ya[0] = xa[0];
        ya[len - 1] = xa[len - 1];
        for (int64_t x = 1; x < len - 1; ++x) {
          REAL uL = xa[x - 1], u = xa[x], uR = xa[x + 1];
          ya[x] = FMA(r, (uR - (REAL)2 * u) + uL, u);
        }
        REAL* t = xa; xa = ya; ya = t;
      }
      for (int64_t i = lo; i < hi; ++i) WB(b + 1, i) = xa[T + (i - lo)];
    }
  }
  for (int64_t i = 0; i < N; ++i) out[i] = WB(nb, i);
#undef WB
  free(off);
  free(W);
  free(ta);
  free(tb_);
  return ORACLE_OK;
}

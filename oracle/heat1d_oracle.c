/*
 * heat1d_oracle.c -- the CPU oracle for the explicit 1D heat-equation update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two never include or
 * link each other.
 *
 * What it computes (Lee & Bhattacharya, "Asynchronous Parallel Computing
 * Algorithm implemented in 1D Heat Equation with CUDA", arXiv:1510.08982):
 *
 *   Section 2, Eq. (eqn:sync):   u_i(k+1) = r u_{i+1}(k) + (1-2r) u_i(k) + r u_{i-1}(k)
 *   Section 2 (Dirichlet ends):  u_1(k) = c_1, u_N(k) = c_2 for every k
 *   Section 3, Eq. (eqn:async):  u_i(k+1) = r u_{i+1}(k*_{i+1}) + (1-2r) u_i(k) + r u_{i-1}(k*_{i-1}),
 *                                k* in {k, k-1, ..., k-q+1}
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *  - Arithmetic order.  The printed kernels of Section 4 evaluate the update as
 *    r*(u[i+1] - 2*u[i] + u[i-1]) + u[i].  The oracle evaluates exactly that,
 *    with the final multiply-add as one fused operation:
 *        v = fma(r, (uR - 2u) + uL, u)
 *    It is compiled with -ffp-contract=off so that no other fusion happens.
 *  - Storage is 0-based: point 0 holds c1 and point N-1 holds cN.  Both are
 *    forced at k = 0 and never updated.
 *  - Asynchrony exists only between processing elements (Section 3: "within a
 *    PE ... no asynchrony").  The points are split into S contiguous segments
 *    (the first N mod S segments get one extra point).  Only a read that crosses
 *    a segment boundary may be delayed.
 *  - The delays are an input: trace[(k*(S-1) + b)*2 + side] for boundary b
 *    (between segments b and b+1).  side 0 is the read made by segment b of its
 *    right neighbour's first point; side 1 is the read made by segment b+1 of
 *    its left neighbour's last point.  Every delay must be < q.  A delay larger
 *    than k is clamped to k (there is no state before k = 0).
 *
 * Error returns: 0 on success, -1 for bad arguments, -5 for a trace entry >= q,
 * -6 when memory cannot be allocated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ETRACE (-5)
#define ORACLE_ENOMEM (-6)

/* Segment split: S contiguous segments of the N points; the first N mod S
 * segments hold one point more than the others.  offsets has S+1 entries. */
int oracle_segments(int64_t N, int64_t S, int64_t* offsets) {
  if (N < 1 || S < 1 || S > N || !offsets) return ORACLE_EINVAL;
  int64_t base = N / S, extra = N % S, pos = 0;
  for (int64_t s = 0; s < S; ++s) {
    offsets[s] = pos;
    pos += base + (s < extra ? 1 : 0);
  }
  offsets[S] = pos;
  return ORACLE_OK;
}

/* The body below is written once for a generic real type and included twice:
 * once for double (f64) and once for float (the exact-order f32 mode). */
#define REAL double
#define FMA fma
#define SUF(name) name##_f64
#include "heat1d_oracle_body.h"
#undef REAL
#undef FMA
#undef SUF

#define REAL float
#define FMA fmaf
#define SUF(name) name##_f32
#include "heat1d_oracle_body.h"
#undef REAL
#undef FMA
#undef SUF

/* Adjoint of the run above (FP64 only): the gradient of
 *     L = 0.5 * sum_i (u_i(K) - u_obs_i)^2
 * with respect to u(0) and r, marched backward through the same delays.
 *
 * Forward, for an interior point i at step k (mathematically, not as rounded):
 *     u_i(k+1) = (1-2r) u_i(k) + r u_{i+1}(k - dR) + r u_{i-1}(k - dL)
 * so with lambda_i(k) = dL/du_i(k):
 *     lambda_i(k)          += (1-2r) lambda_i(k+1)
 *     lambda_{i+1}(k - dR) += r lambda_i(k+1)
 *     lambda_{i-1}(k - dL) += r lambda_i(k+1)
 *     dL/dr                += lambda_i(k+1) * ((u_{i+1}(k-dR) - 2 u_i(k)) + u_{i-1}(k-dL))
 * with lambda(K) = u(K) - u_obs on the interior.  The end points are constants,
 * so their gradient is zero.  The full forward trajectory and the full lambda
 * history are stored: this is only meant for test sizes.  dL/dr and the loss
 * are summed with Kahan compensation.  trace == NULL means the synchronous
 * run (every delay 0).
 */
int oracle_adjoint_f64(int64_t N, double r, double c1, double cN, int64_t S, int q,
                       const double* u0, int64_t K, const uint8_t* trace, const double* u_obs,
                       double* grad_u0, double* grad_r, double* loss) {
  if (N < 3 || K < 0 || !u0 || !u_obs || !grad_u0 || !grad_r || !loss) return ORACLE_EINVAL;
  if (trace && (S < 1 || S > N || q < 1)) return ORACLE_EINVAL;
  if (!trace) { S = 1; q = 1; }
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  int64_t* seg = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  double* U = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(K + 1));
  double* lam = (double*)calloc((size_t)N * (size_t)(K + 1), sizeof(double));
  if (!off || !seg || !U || !lam) { free(off); free(seg); free(U); free(lam); return ORACLE_ENOMEM; }
  oracle_segments(N, S, off);
  for (int64_t s = 0; s < S; ++s)
    for (int64_t i = off[s]; i < off[s + 1]; ++i) seg[i] = s;
  if (trace) {
    for (int64_t j = 0; j < K * (S - 1) * 2; ++j)
      if (trace[j] >= q) { free(off); free(seg); free(U); free(lam); return ORACLE_ETRACE; }
  }
#define UU(t, i) U[(size_t)(t) * (size_t)N + (size_t)(i)]
#define LL(t, i) lam[(size_t)(t) * (size_t)N + (size_t)(i)]
  /* Forward pass: store every state. */
  for (int64_t i = 0; i < N; ++i) UU(0, i) = u0[i];
  UU(0, 0) = c1;
  UU(0, N - 1) = cN;
  for (int64_t k = 0; k < K; ++k) {
    UU(k + 1, 0) = c1;
    UU(k + 1, N - 1) = cN;
    for (int64_t i = 1; i < N - 1; ++i) {
      int64_t tL = k, tR = k;
      if (seg[i - 1] != seg[i]) {
        int64_t d = trace[(k * (S - 1) + seg[i - 1]) * 2 + 1];
        tL = k - (d < k ? d : k);
      }
      if (seg[i + 1] != seg[i]) {
        int64_t d = trace[(k * (S - 1) + seg[i]) * 2 + 0];
        tR = k - (d < k ? d : k);
      }
      double uL = UU(tL, i - 1), uR = UU(tR, i + 1), u = UU(k, i);
      UU(k + 1, i) = fma(r, (uR - 2.0 * u) + uL, u);
    }
  }
  /* Loss and terminal adjoint. */
  double ls = 0.0, lc = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double e = UU(K, i) - u_obs[i];
    double y = 0.5 * e * e - lc, t = ls + y;
    lc = (t - ls) - y;
    ls = t;
    if (i > 0 && i < N - 1) LL(K, i) = e;
  }
  /* Backward pass. */
  double gs = 0.0, gc = 0.0;
  for (int64_t k = K - 1; k >= 0; --k) {
    for (int64_t i = 1; i < N - 1; ++i) {
      double g = LL(k + 1, i);
      int64_t tL = k, tR = k;
      if (seg[i - 1] != seg[i]) {
        int64_t d = trace[(k * (S - 1) + seg[i - 1]) * 2 + 1];
        tL = k - (d < k ? d : k);
      }
      if (seg[i + 1] != seg[i]) {
        int64_t d = trace[(k * (S - 1) + seg[i]) * 2 + 0];
        tR = k - (d < k ? d : k);
      }
      LL(k, i) += (1.0 - 2.0 * r) * g;
      LL(tR, i + 1) += r * g;
      LL(tL, i - 1) += r * g;
      double du = (UU(tR, i + 1) - 2.0 * UU(k, i)) + UU(tL, i - 1);
      double y = g * du - gc, t = gs + y;
      gc = (t - gs) - y;
      gs = t;
    }
  }
  for (int64_t i = 0; i < N; ++i) grad_u0[i] = (i > 0 && i < N - 1) ? LL(0, i) : 0.0;
  *grad_r = gs;
  *loss = ls;
#undef UU
#undef LL
  free(off);
  free(seg);
  free(U);
  free(lam);
  return ORACLE_OK;
}

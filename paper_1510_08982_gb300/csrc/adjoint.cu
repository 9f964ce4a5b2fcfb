// adjoint.cu -- gradient of the terminal misfit L = 0.5 ||u(K) - u_obs||^2
// with respect to u(0) and r, for the synchronous run (Section 2, Eq.
// (eqn:sync)) and for a replayed asynchronous run (Section 3, Eq.
// (eqn:async) driven by a recorded delay trace).
//
// Forward, per interior point and step (mathematically):
//   u_i(k+1) = (1-2r) u_i(k) + r u_{i+1}(k - dR) + r u_{i-1}(k - dL)
// where dR, dL are the trace's delays on reads that cross a segment boundary
// (0 elsewhere, and clamped to k).  With lambda(k) = dL/du(k):
//   lambda(K)            = u(K) - u_obs on the interior, 0 at the ends
//   lambda_i(k)          += (1-2r) lambda_i(k+1)
//   lambda_{i+1}(k - dR) += r lambda_i(k+1)
//   lambda_{i-1}(k - dL) += r lambda_i(k+1)
//   dL/dr                += lambda_i(k+1) ((u_{i+1}(k-dR) - 2 u_i(k)) + u_{i-1}(k-dL))
// A read made with delay d > 0 becomes, in the backward march, a contribution
// to an earlier time level that has not been reached yet: it is parked in a
// ring of q+1 pending sums per boundary point and added when the march gets
// there.  Contributions with d = 0 are gathered directly, so a backward step
// is a gather like the forward stencil.
//
// Memory: the forward pass keeps a checkpoint every C steps (the full state
// plus the last q values of every boundary point, which delayed reads may
// need); the backward pass recomputes each interval from its checkpoint into
// a workspace of C+1 states and then marches lambda back through it.
//
// Each step is one launch over all points of all rods (the backward march
// needs every point of step k before any of step k-1).  lambda is stored and
// stepped in the state's precision; the loss and dL/dr are summed in FP64
// (an FP32 run adds a warp's products in FP32 first).  Every reduction is
// deterministic: fixed per-block partials with compensated sums, added in a
// fixed order at the end.
#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

constexpr int kAdjThreads = 256;
// A block walks kAdjThreads * this many points of one rod: 16 in FP64, 32 in
// FP32 (measured: FP32 runs gain from the longer walk, FP64 runs lose).
template <typename real>
constexpr int adj_points_per_thread() { return sizeof(real) == 4 ? 32 : 16; }

struct AdjGeom {
  int64_t nrods, N;
  int S;          // segments per rod
  int64_t seg_base, seg_extra;  // N / S and N mod S
  int q, Q;       // delay window, pending ring length (q+1)
  int64_t bpr;    // blocks per rod
  int64_t span;   // points per block (a block never straddles two rods)
  const double* r;
  const double* c1;
  const double* cN;
  const float* rf;   // the same coefficients rounded to FP32 (read by FP32 runs: no conversions on the FP64 pipe)
  const float* c1f;
  const float* cNf;
  const uint8_t* trace;  // [rod][K][S-1][2] or null (synchronous)
  int64_t K;
};

// Rod coefficients in the run's precision.
template <typename real>
struct Coefs;
template <>
struct Coefs<double> {
  __device__ static double r(const AdjGeom& g, int64_t rod) { return g.r[rod]; }
  __device__ static double c1(const AdjGeom& g, int64_t rod) { return g.c1[rod]; }
  __device__ static double cN(const AdjGeom& g, int64_t rod) { return g.cN[rod]; }
};
template <>
struct Coefs<float> {
  __device__ static float r(const AdjGeom& g, int64_t rod) { return g.rf[rod]; }
  __device__ static float c1(const AdjGeom& g, int64_t rod) { return g.c1f[rod]; }
  __device__ static float cN(const AdjGeom& g, int64_t rod) { return g.cNf[rod]; }
};

// Segment geometry of a rod (the first N mod S segments one point longer),
// from seg_base = N / S and seg_extra = N mod S computed on the host: no
// 64-bit division on the device (it costs hundreds of instructions), and a
// 32-bit one where the operands fit.
__device__ __forceinline__ int64_t udiv(int64_t a, int64_t b) {  // a >= 0, b > 0
  return (a <= 0xffffffffLL && b <= 0xffffffffLL)
             ? static_cast<int64_t>(static_cast<uint32_t>(a) / static_cast<uint32_t>(b))
             : a / b;
}
__device__ __forceinline__ int seg_of(int64_t i, const AdjGeom& g) {
  const int64_t big = g.seg_extra * (g.seg_base + 1);
  return static_cast<int>(i < big ? udiv(i, g.seg_base + 1) : g.seg_extra + udiv(i - big, g.seg_base));
}
__device__ __forceinline__ int64_t seg_start(int s, const AdjGeom& g) {
  return s * g.seg_base + (s < g.seg_extra ? s : g.seg_extra);
}

// The segment of a thread's points as they increase: one division for the
// first point, then comparisons only (a thread's points are kAdjThreads
// apart, far less than a segment is long in the workloads of interest, and
// any gap is walked).
struct SegTrack {
  int s;
  int64_t lo, hi;  // the current segment's points [lo, hi)
  __device__ __forceinline__ void init(int64_t i, const AdjGeom& g) {
    s = seg_of(i, g);
    lo = seg_start(s, g);
    hi = seg_start(s + 1, g);
  }
  __device__ __forceinline__ void advance(int64_t i, const AdjGeom& g) {
    while (i >= hi) {
      ++s;
      lo = hi;
      hi = seg_start(s + 1, g);
    }
  }
};

__device__ __forceinline__ int delay_at(const AdjGeom& g, int64_t rod, int64_t k, int b, int side) {
  const int d = g.trace[((rod * g.K + k) * (g.S - 1) + b) * 2 + side];
  return static_cast<int>(d < k ? d : k);
}

// Edge history: for each time t of the current interval a row of
// [rod][S-1][2] values: side 0 = first point of segment b+1, side 1 = last
// point of segment b.  Row of time t is t - t0 (t0 = first time held).
template <typename real>
__device__ __forceinline__ real* eh_row(real* eh, const AdjGeom& g, int64_t row) {
  return eh + row * g.nrods * (g.S - 1) * 2;
}

// Sets the Dirichlet ends of every rod of a state row.
template <typename real>
__global__ void adj_force_ends(AdjGeom g, real* u) {
  const int64_t rod = blockIdx.x * blockDim.x + threadIdx.x;
  if (rod >= g.nrods) return;
  u[rod * g.N] = Coefs<real>::c1(g, rod);
  u[rod * g.N + g.N - 1] = Coefs<real>::cN(g, rod);
}

// Writes the boundary points of state row `u` (all rods) into history row.
template <typename real>
__global__ void adj_edge_gather(AdjGeom g, const real* u, real* eh_dst) {
  const int64_t n = g.nrods * (g.S - 1);
  for (int64_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
    const int64_t rod = x / (g.S - 1);
    const int b = static_cast<int>(x % (g.S - 1));
    const int64_t first = seg_start(b + 1, g);
    eh_dst[x * 2 + 0] = u[rod * g.N + first];
    eh_dst[x * 2 + 1] = u[rod * g.N + first - 1];
  }
}

// One forward step k -> k+1 for every point of every rod (same arithmetic as
// the persistent kernels).  Delayed reads come from the edge history.
template <typename real>
__global__ void __launch_bounds__(kAdjThreads) adj_fwd_step(AdjGeom g, int64_t k, const real* __restrict__ u,
                                                            real* __restrict__ out, real* eh, int64_t t0) {
  const int64_t rod = blockIdx.x / g.bpr;
  const int64_t b0 = (blockIdx.x % g.bpr) * g.span;
  const int64_t b1 = min(b0 + g.span, g.N);
  const real* ur = u + rod * g.N;
  real* orow = out + rod * g.N;
  const real r = Coefs<real>::r(g, rod);
  const real one = static_cast<real>(g.N > 0);
  SegTrack sg{};
  if (g.trace) sg.init(b0 + threadIdx.x, g);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kAdjThreads) {
    bool first = false, last = false;  // the segment's first / last point
    int s = 0;
    if (g.trace) {
      sg.advance(i, g);
      s = sg.s;
      first = s > 0 && i == sg.lo;
      last = s + 1 < g.S && i == sg.hi - 1;
    }
    real v;
    if (i == 0) {
      v = Coefs<real>::c1(g, rod);
    } else if (i == g.N - 1) {
      v = Coefs<real>::cN(g, rod);
    } else {
      real uL = ur[i - 1], uR = ur[i + 1];
      if (first) {
        const int d = delay_at(g, rod, k, s - 1, 1);
        if (d > 0) uL = eh_row(eh, g, k - d - t0)[(rod * (g.S - 1) + (s - 1)) * 2 + 1];
      }
      if (last) {
        const int d = delay_at(g, rod, k, s, 0);
        if (d > 0) uR = eh_row(eh, g, k - d - t0)[(rod * (g.S - 1) + s) * 2 + 0];
      }
      v = ftcs(r, one, uL, ur[i], uR);
    }
    orow[i] = v;
    if (first || last) {  // boundary points of time k+1 into the history
      real* row = eh_row(eh, g, k + 1 - t0);
      if (first) row[(rod * (g.S - 1) + (s - 1)) * 2 + 0] = v;
      if (last) row[(rod * (g.S - 1) + s) * 2 + 1] = v;
    }
  }
}

template <typename real>
struct Vec16T;
template <>
struct Vec16T<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16T<double> {
  using type = double2;
  static constexpr int n = 2;
};

// The segment-boundary points of a block [b0, b1) of one rod: candidate j is
// the first (even j) or last (odd j) point of segment s0 + j/2, where s0 is
// the segment of b0.  Returns false when candidate j is not such a point of
// this block; a one-point segment is handled once, as its first point.
__device__ __forceinline__ bool boundary_point(const AdjGeom& g, int s0, int j, int64_t b0, int64_t b1, int64_t& i,
                                               int& s, bool& first, bool& last) {
  s = s0 + j / 2;
  const int64_t lo = seg_start(s, g), hi = seg_start(s + 1, g);
  i = (j & 1) ? hi - 1 : lo;
  if ((j & 1) && i == lo) return false;
  first = i == lo && s > 0;
  last = i == hi - 1 && s + 1 < g.S;
  return (first || last) && i >= b0 && i < b1;
}
__device__ __forceinline__ int boundary_candidates(const AdjGeom& g, int64_t b0, int64_t b1, int& s0) {
  s0 = seg_of(b0, g);
  return 2 * (seg_of(b1 - 1, g) - s0 + 1);
}

// Forward step of a replay at the block's segment-boundary points: the
// delayed neighbour values from the edge history (the synchronous sweep
// used the current ones), and the new values into the history row k+1.
template <typename real>
__device__ void fwd_fixup(const AdjGeom& g, int64_t k, const real* ur, real* orow, real* eh, int64_t t0, int64_t rod,
                          int64_t b0, int64_t b1, real r, real one, real c1, real cN) {
  int s0 = 0;
  const int nc = boundary_candidates(g, b0, b1, s0);
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    int64_t i;
    int s;
    bool first, last;
    if (!boundary_point(g, s0, j, b0, b1, i, s, first, last)) continue;
    real v;
    if (i == 0) {
      v = c1;
    } else if (i == g.N - 1) {
      v = cN;
    } else {
      real uL = ur[i - 1], uR = ur[i + 1];
      if (first) {
        const int d = delay_at(g, rod, k, s - 1, 1);
        if (d > 0) uL = eh_row(eh, g, k - d - t0)[(rod * (g.S - 1) + (s - 1)) * 2 + 1];
      }
      if (last) {
        const int d = delay_at(g, rod, k, s, 0);
        if (d > 0) uR = eh_row(eh, g, k - d - t0)[(rod * (g.S - 1) + s) * 2 + 0];
      }
      v = ftcs(r, one, uL, ur[i], uR);
    }
    orow[i] = v;
    real* row = eh_row(eh, g, k + 1 - t0);  // boundary points of time k+1 into the history
    if (first) row[(rod * (g.S - 1) + (s - 1)) * 2 + 0] = v;
    if (last) row[(rod * (g.S - 1) + s) * 2 + 1] = v;
  }
}

// The same forward step with 16-byte vectors: a thread updates VN consecutive
// points per pass and takes its two outer neighbours from the adjacent lanes
// (lane 0, lane 31 and a lane whose right neighbour is past the block load
// theirs).  Same arithmetic, delayed reads and history writes as adj_fwd_step.
// The next pass's vector is loaded before the current one is computed; a
// vector whose points are all interior (and, in a replay, none a segment's
// first or last) takes the plain stencil.  Requires N to be a multiple of VN,
// so that every rod row and every block starts on a 16-byte boundary and no
// vector straddles the end of a block.
template <typename real, bool kTrace>
__global__ void __launch_bounds__(kAdjThreads) adj_fwd_step_vec(AdjGeom g, int64_t k, const real* __restrict__ u,
                                                                real* __restrict__ out, real* eh, int64_t t0) {
  using V = typename Vec16T<real>::type;
  constexpr int VN = Vec16T<real>::n;
  constexpr bool kInline = kTrace && sizeof(real) == 8;  // replay: delayed reads inside the sweep (FP64)
  constexpr bool kFix = kTrace && sizeof(real) == 4;     // replay: synchronous sweep, then fwd_fixup (FP32)
  const unsigned bpr = static_cast<unsigned>(g.bpr);
  const unsigned rod32 = blockIdx.x / bpr;
  const int64_t rod = rod32;
  const int64_t b0 = static_cast<int64_t>(blockIdx.x - rod32 * bpr) * g.span;
  const int64_t b1 = min(b0 + g.span, g.N);
  const int64_t N = g.N;
  const real* ur = u + rod * N;
  real* orow = out + rod * N;
  const real r = Coefs<real>::r(g, rod);
  const real one = static_cast<real>(g.N > 0);
  const real c1 = Coefs<real>::c1(g, rod), cN = Coefs<real>::cN(g, rod);
  const int lane = threadIdx.x & 31;
  const int passes = static_cast<int>(g.span / (static_cast<int64_t>(kAdjThreads) * VN));
  constexpr int64_t stride = static_cast<int64_t>(kAdjThreads) * VN;
  SegTrack sg{};
  if (kInline) sg.init(min(b0 + static_cast<int64_t>(threadIdx.x) * VN, N - 1), g);
  int64_t i0 = b0 + static_cast<int64_t>(threadIdx.x) * VN;
  V wn{};
  if (i0 < b1) wn = *reinterpret_cast<const V*>(ur + i0);
  for (int pass = 0; pass < passes; ++pass, i0 += stride) {  // warp-uniform trip count (shuffles)
    const bool active = i0 < b1;
    real x[VN];
    {
      const real* ws = reinterpret_cast<const real*>(&wn);
#pragma unroll
      for (int e = 0; e < VN; ++e) x[e] = ws[e];
    }
    if (pass + 1 < passes && i0 + stride < b1) wn = *reinterpret_cast<const V*>(ur + i0 + stride);
    real left = __shfl_up_sync(0xffffffffu, x[VN - 1], 1);
    real right = __shfl_down_sync(0xffffffffu, x[0], 1);
    if (!active) continue;
    if (lane == 0) left = i0 > 0 ? ur[i0 - 1] : static_cast<real>(0);
    if ((lane == 31 || i0 + VN >= b1) && i0 + VN < N) right = ur[i0 + VN];
    real y[VN];
    bool plain = i0 >= 1 && i0 + VN <= N - 1;
    if (kInline && plain) {
      sg.advance(i0, g);
      plain = i0 > sg.lo && i0 + VN < sg.hi;
    }
    if (plain) {
#pragma unroll
      for (int e = 0; e < VN; ++e) y[e] = ftcs(r, one, e > 0 ? x[e - 1] : left, x[e], e + 1 < VN ? x[e + 1] : right);
    } else {
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        const int64_t i = i0 + e;
        bool first = false, last = false;
        int s = 0;
        if (kInline) {
          sg.advance(i, g);
          s = sg.s;
          first = s > 0 && i == sg.lo;
          last = s + 1 < g.S && i == sg.hi - 1;
        }
        real v;
        if (i == 0) {
          v = c1;
        } else if (i == N - 1) {
          v = cN;
        } else {
          real uL = e > 0 ? x[e - 1] : left;
          real uR = e + 1 < VN ? x[e + 1] : right;
          if (first) {
            const int d = delay_at(g, rod, k, s - 1, 1);
            if (d > 0) uL = eh_row(eh, g, k - d - t0)[(rod * (g.S - 1) + (s - 1)) * 2 + 1];
          }
          if (last) {
            const int d = delay_at(g, rod, k, s, 0);
            if (d > 0) uR = eh_row(eh, g, k - d - t0)[(rod * (g.S - 1) + s) * 2 + 0];
          }
          v = ftcs(r, one, uL, x[e], uR);
        }
        y[e] = v;
        if (first || last) {  // boundary points of time k+1 into the history
          real* row = eh_row(eh, g, k + 1 - t0);
          if (first) row[(rod * (g.S - 1) + (s - 1)) * 2 + 0] = v;
          if (last) row[(rod * (g.S - 1) + s) * 2 + 1] = v;
        }
      }
    }
    V w;
    real* ws = reinterpret_cast<real*>(&w);
#pragma unroll
    for (int e = 0; e < VN; ++e) ws[e] = y[e];
    *reinterpret_cast<V*>(orow + i0) = w;
  }
  if (kFix) {  // the block's segment-boundary points, redone with their delayed reads
    __syncthreads();
    fwd_fixup<real>(g, k, ur, orow, eh, t0, rod, b0, b1, r, one, c1, cN);
  }
}

// Block-wide sum of one double per thread in a fixed order: warp shuffles,
// then the warps' sums in warp order.
__device__ double block_sum(double x, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFullMask, x, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int j = 0; j < kAdjThreads / 32; ++j) s += red[j];
  __syncthreads();
  return s;  // valid in thread 0
}

// The r-gradient partial of a block: a thread's product sum `acc` plus its
// FP64 delayed-read terms.  FP64 runs sum both in FP64.  FP32 runs sum the
// products of a warp in FP32 and the warps' sums in FP64 (the shuffled
// additions of a warp would otherwise be FP64-pipe work for every lane); the
// delayed-read terms, present only in replays, stay FP64.
template <bool kTrace>
__device__ double block_sum_acc(double acc, double terms, double* red) {
  return block_sum(acc + terms, red);
}
template <bool kTrace>
__device__ double block_sum_acc(float acc, double terms, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFullMask, acc, o);
  if (kTrace) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) terms += __shfl_down_sync(kFullMask, terms, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = static_cast<double>(acc) + terms;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int j = 0; j < kAdjThreads / 32; ++j) s += red[j];
  __syncthreads();
  return s;  // valid in thread 0
}

// Compensated accumulation of one partial per block.
__device__ void kahan_add(double* sum, double* comp, double x) {
  const double y = x - *comp;
  const double t = *sum + y;
  *comp = (t - *sum) - y;
  *sum = t;
}

// The backward step's arithmetic in the run's precision: lambda is stored and
// stepped in the state's type.  FP64: the additions are issued as fused
// multiply-adds by a run-time 1.0 (exact, the same rounded sums; the FP64 pipe
// sustains DFMA at a higher rate than DADD).  FP32: FP32 operations.
__device__ __forceinline__ double adj_lap(double one, double lc, double ll, double lr) {
  return __fma_rn(one, __fma_rn(-2.0, lc, lr), ll);
}
__device__ __forceinline__ float adj_lap(float, float lc, float ll, float lr) {
  return __fadd_rn(__fmaf_rn(-2.0f, lc, lr), ll);
}
__device__ __forceinline__ double adj_new(double one, double r, double tl, double lc, double pending) {
  return __fma_rn(one, __fma_rn(r, tl, lc), pending);
}
__device__ __forceinline__ float adj_new(float, float r, float tl, float lc, float pending) {
  return __fadd_rn(__fmaf_rn(r, tl, lc), pending);
}
// The update of a point with nothing pending (no delayed read involved).
__device__ __forceinline__ double adj_new0(double r, double t, double lc) { return __fma_rn(r, t, lc); }
__device__ __forceinline__ float adj_new0(float r, float t, float lc) { return __fmaf_rn(r, t, lc); }
// dL/dr products u_i t_i of a thread: FP64 runs sum them in FP64; FP32 runs
// sum a thread's products (its points of one block) in FP32, then a warp's
// thread sums in FP32 (block_sum_acc), and add the warp sums to the FP64
// partials, so that the FP64 pipe is not the bound of an FP32 run.
__device__ __forceinline__ double adj_prod(double u, double t, double acc) { return __fma_rn(u, t, acc); }
__device__ __forceinline__ float adj_prod(float u, float t, float acc) { return __fmaf_rn(u, t, acc); }
// A delayed-read term of dL/dr: into the FP64 sum (FP64 runs keep one sum, in
// point order).
__device__ __forceinline__ void adj_term(double& acc, double& /*terms*/, double x) { acc += x; }
__device__ __forceinline__ void adj_term(float& /*acc*/, double& terms, double x) { terms += x; }

// lambda(K) = u(K) - u_obs on the interior; per-block loss partials.
// With `cotangent` set, uobs is dL/du(K) itself and the loss is reported 0.
template <typename real>
__global__ void __launch_bounds__(kAdjThreads) adj_init(AdjGeom g, const real* __restrict__ uK,
                                                        const double* __restrict__ uobs, real* __restrict__ lam,
                                                        double* loss_part, int cotangent) {
  __shared__ double red[kAdjThreads / 32];
  const int64_t rod = blockIdx.x / g.bpr;
  const int64_t b0 = (blockIdx.x % g.bpr) * g.span;
  const int64_t b1 = min(b0 + g.span, g.N);
  double e2 = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kAdjThreads) {
    const int64_t x = rod * g.N + i;
    const double e = cotangent ? uobs[x] : static_cast<double>(uK[x]) - uobs[x];
    if (!cotangent) e2 += 0.5 * e * e;
    lam[x] = static_cast<real>((i > 0 && i < g.N - 1) ? e : 0.0);
  }
  const double s = block_sum(e2, red);
  if (threadIdx.x == 0) loss_part[blockIdx.x] = s;
}

// One backward step: lambda(k) from lambda(k+1), with u(k) (row `u`) and the
// edge history for delayed reads; dL/dr partials per block.
//
// With lambda extended by zeros beyond the interior, t_i = (lambda_{i+1} -
// 2 lambda_i) + lambda_{i-1} serves both halves of the step:
//   - lambda_i(k) = lambda_i(k+1) + r t_i, minus the terms of neighbours whose
//     read of u_i was delayed (those arrive later through the pending ring);
//   - by summation by parts, sum_{interior i} lambda_i ((u_{i+1} - 2u_i) +
//     u_{i-1}) = sum_{all i} u_i t_i, so dL/dr gains u_i(k) t_i per point,
//     plus lambda_i (u_{i+-1}(k-d) - u_{i+-1}(k)) where point i read a
//     neighbour with delay d > 0.
template <typename real>
__global__ void __launch_bounds__(kAdjThreads) adj_bwd_step(AdjGeom g, int64_t k, const real* __restrict__ lin,
                                                            real* __restrict__ lout, const real* __restrict__ u,
                                                            const real* eh, int64_t t0, double* pend,
                                                            double* gr_sum, double* gr_comp) {
  __shared__ double red[kAdjThreads / 32];
  const int64_t rod = blockIdx.x / g.bpr;
  const int64_t b0 = (blockIdx.x % g.bpr) * g.span;
  const int64_t b1 = min(b0 + g.span, g.N);
  real acc = 0;          // products u_i t_i (and, in FP64, the delayed-read terms)
  double contrib = 0.0;  // FP32: the delayed-read terms
  const real one = static_cast<real>(g.N > 0);
  const real zero = 0;
  SegTrack sg{};
  if (g.trace) sg.init(b0 + threadIdx.x, g);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kAdjThreads) {
    const int64_t base = rod * g.N;
    const int64_t N = g.N;
    const real lc = (i >= 1 && i <= N - 2) ? lin[base + i] : zero;
    const real ll = (i - 1 >= 1 && i - 1 <= N - 2) ? lin[base + i - 1] : zero;
    const real lr = (i + 1 >= 1 && i + 1 <= N - 2) ? lin[base + i + 1] : zero;
    const real* ur = u + base;
    const real t = adj_lap(one, lc, ll, lr);
    acc = adj_prod(ur[i], t, acc);
    if (i == 0 || i == N - 1) {
      lout[base + i] = zero;
    } else {
      const real r = Coefs<real>::r(g, rod);
      real tl = t;        // t without the neighbour terms that arrive delayed
      real pending = 0;
      if (g.trace) {
        sg.advance(i, g);
        const int s = sg.s;
        const bool first = s > 0 && i == sg.lo;
        const bool last = s + 1 < g.S && i == sg.hi - 1;
        if (first || last) {
          double* prow = pend + (k % g.Q) * g.nrods * (g.S - 1) * 2;
          if (first) {
            double* p = prow + (rod * (g.S - 1) + (s - 1)) * 2 + 0;  // parked from i-1's delayed right reads
            pending += static_cast<real>(*p);
            *p = 0.0;
            if (delay_at(g, rod, k, s - 1, 0) > 0) tl -= ll;  // i-1 read u_i late: its term is parked
            const int dL = delay_at(g, rod, k, s - 1, 1);   // this point's own left read
            if (dL > 0) {
              const double uLd = static_cast<double>(eh_row(eh, g, k - dL - t0)[(rod * (g.S - 1) + (s - 1)) * 2 + 1]);
              adj_term(acc, contrib, static_cast<double>(lc) * (uLd - static_cast<double>(ur[i - 1])));
              pend[((k - dL) % g.Q) * g.nrods * (g.S - 1) * 2 + (rod * (g.S - 1) + (s - 1)) * 2 + 1] += r * lc;
            }
          }
          if (last) {
            double* p = prow + (rod * (g.S - 1) + s) * 2 + 1;  // parked from i+1's delayed left reads
            pending += static_cast<real>(*p);
            *p = 0.0;
            if (delay_at(g, rod, k, s, 1) > 0) tl -= lr;    // i+1 read u_i late
            const int dR = delay_at(g, rod, k, s, 0);       // this point's own right read
            if (dR > 0) {
              const double uRd = static_cast<double>(eh_row(eh, g, k - dR - t0)[(rod * (g.S - 1) + s) * 2 + 0]);
              adj_term(acc, contrib, static_cast<double>(lc) * (uRd - static_cast<double>(ur[i + 1])));
              pend[((k - dR) % g.Q) * g.nrods * (g.S - 1) * 2 + (rod * (g.S - 1) + s) * 2 + 0] += r * lc;
            }
          }
        }
      }
      lout[base + i] = adj_new(one, r, tl, lc, pending);
    }
  }
  const double bs = block_sum(static_cast<double>(acc) + contrib, red);
  if (threadIdx.x == 0) kahan_add(gr_sum + blockIdx.x, gr_comp + blockIdx.x, bs);
}

// Backward step of a replay at the block's segment-boundary points, as in
// adj_bwd_step: the neighbour terms whose reads were delayed leave t and come
// back through the pending ring; this point's own delayed reads add their
// dL/dr terms and park r * lambda_i for the earlier level they came from.
template <typename real>
__device__ void bwd_fixup(const AdjGeom& g, int64_t k, const real* lin, real* lout, const real* ur, const real* eh,
                          int64_t t0, double* pend, int64_t rod, int64_t base, int64_t b0, int64_t b1, real r,
                          real one, real& acc, double& contrib) {
  const int64_t N = g.N;
  const real zero = 0;
  int s0 = 0;
  const int nc = boundary_candidates(g, b0, b1, s0);
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    int64_t i;
    int s;
    bool first, last;
    if (!boundary_point(g, s0, j, b0, b1, i, s, first, last)) continue;
    if (i == 0 || i == N - 1) continue;  // Dirichlet ends: lambda stays 0
    const real lc = lin[base + i];
    const real ll = i - 1 >= 1 ? lin[base + i - 1] : zero;
    const real lr = i + 1 <= N - 2 ? lin[base + i + 1] : zero;
    real tl = adj_lap(one, lc, ll, lr);  // t without the neighbour terms that arrive delayed
    real pending = 0;
    double* prow = pend + (k % g.Q) * g.nrods * (g.S - 1) * 2;
    if (first) {
      double* p = prow + (rod * (g.S - 1) + (s - 1)) * 2 + 0;  // parked from i-1's delayed right reads
      pending += static_cast<real>(*p);
      *p = 0.0;
      if (delay_at(g, rod, k, s - 1, 0) > 0) tl -= ll;  // i-1 read u_i late: its term is parked
      const int dL = delay_at(g, rod, k, s - 1, 1);   // this point's own left read
      if (dL > 0) {
        const double uLd = static_cast<double>(eh_row(eh, g, k - dL - t0)[(rod * (g.S - 1) + (s - 1)) * 2 + 1]);
        adj_term(acc, contrib, static_cast<double>(lc) * (uLd - static_cast<double>(ur[i - 1])));
        pend[((k - dL) % g.Q) * g.nrods * (g.S - 1) * 2 + (rod * (g.S - 1) + (s - 1)) * 2 + 1] += r * lc;
      }
    }
    if (last) {
      double* p = prow + (rod * (g.S - 1) + s) * 2 + 1;  // parked from i+1's delayed left reads
      pending += static_cast<real>(*p);
      *p = 0.0;
      if (delay_at(g, rod, k, s, 1) > 0) tl -= lr;    // i+1 read u_i late
      const int dR = delay_at(g, rod, k, s, 0);       // this point's own right read
      if (dR > 0) {
        const double uRd = static_cast<double>(eh_row(eh, g, k - dR - t0)[(rod * (g.S - 1) + s) * 2 + 0]);
        adj_term(acc, contrib, static_cast<double>(lc) * (uRd - static_cast<double>(ur[i + 1])));
        pend[((k - dR) % g.Q) * g.nrods * (g.S - 1) * 2 + (rod * (g.S - 1) + s) * 2 + 0] += r * lc;
      }
    }
    lout[base + i] = adj_new(one, r, tl, lc, pending);
  }
}

// The same backward step, VN points per thread and pass: lambda and u move as
// 16-byte vectors, the next pass's vectors are loaded before the current ones
// are used, and the outer lambda neighbours come from the adjacent lanes (lane
// 0, lane 31 and a lane whose right neighbour is past the block load theirs).
// A vector whose points and neighbours are all interior (and, in a replay,
// none of whose points is a segment's first or last) takes the plain
// transposed stencil with nothing pending; the others follow adj_bwd_step
// point by point (delayed-read corrections, pending ring).  The r-gradient
// partial of a block is summed in a fixed order (each thread's points in
// order, then block_sum), so it does not depend on the checkpoint interval.
// Requires N to be a multiple of VN.
template <typename real, bool kTrace>
__global__ void __launch_bounds__(kAdjThreads, 4) adj_bwd_step_vec(AdjGeom g, int64_t k, const real* __restrict__ lin,
                                                                real* __restrict__ lout, const real* __restrict__ u,
                                                                const real* eh, int64_t t0, double* pend,
                                                                double* gr_sum, double* gr_comp) {
  using V = typename Vec16T<real>::type;
  constexpr int VN = Vec16T<real>::n;
  constexpr bool kInline = kTrace && sizeof(real) == 8;  // replay: delayed reads inside the sweep (FP64)
  constexpr bool kFix = kTrace && sizeof(real) == 4;     // replay: synchronous sweep, then bwd_fixup (FP32)
  __shared__ double red[kAdjThreads / 32];
  const unsigned bpr = static_cast<unsigned>(g.bpr);
  const unsigned rod32 = blockIdx.x / bpr;
  const int64_t rod = rod32;
  const int64_t b0 = static_cast<int64_t>(blockIdx.x - rod32 * bpr) * g.span;
  const int64_t b1 = min(b0 + g.span, g.N);
  const int64_t N = g.N;
  const int64_t base = rod * N;
  const real* ur = u + base;
  const real r = Coefs<real>::r(g, rod);
  const real one = static_cast<real>(g.N > 0);
  const real zero = 0;
  const int lane = threadIdx.x & 31;
  const int passes = static_cast<int>(g.span / (static_cast<int64_t>(kAdjThreads) * VN));
  constexpr int64_t stride = static_cast<int64_t>(kAdjThreads) * VN;
  real acc = 0;          // products u_i t_i (and, in FP64, the delayed-read terms)
  double contrib = 0.0;  // FP32: the delayed-read terms
  SegTrack sg{};
  if (kInline) sg.init(min(b0 + static_cast<int64_t>(threadIdx.x) * VN, N - 1), g);
  int64_t i0 = b0 + static_cast<int64_t>(threadIdx.x) * VN;
  V ln{}, un{};
  if (i0 < b1) {
    ln = *reinterpret_cast<const V*>(lin + base + i0);
    un = *reinterpret_cast<const V*>(ur + i0);
  }
  for (int pass = 0; pass < passes; ++pass, i0 += stride) {  // warp-uniform trip count (shuffles)
    const bool active = i0 < b1;
    real L[VN], U[VN];
    {
      const real* lv = reinterpret_cast<const real*>(&ln);
      const real* uv = reinterpret_cast<const real*>(&un);
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        L[e] = lv[e];
        U[e] = uv[e];
      }
    }
    if (pass + 1 < passes && i0 + stride < b1) {
      ln = *reinterpret_cast<const V*>(lin + base + i0 + stride);
      un = *reinterpret_cast<const V*>(ur + i0 + stride);
    }
    real lleft = __shfl_up_sync(0xffffffffu, L[VN - 1], 1);
    real lright = __shfl_down_sync(0xffffffffu, L[0], 1);
    if (!active) continue;
    if (lane == 0) lleft = i0 > 0 ? lin[base + i0 - 1] : zero;
    if ((lane == 31 || i0 + VN >= b1) && i0 + VN < N) lright = lin[base + i0 + VN];
    real out[VN];
    bool plain = i0 >= 2 && i0 + VN <= N - 2;  // the points and their neighbours interior
    if (kInline && plain) {
      sg.advance(i0, g);
      plain = i0 > sg.lo && i0 + VN < sg.hi;
    }
    if (plain) {
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        const real t = adj_lap(one, L[e], e > 0 ? L[e - 1] : lleft, e + 1 < VN ? L[e + 1] : lright);
        acc = adj_prod(U[e], t, acc);
        out[e] = adj_new0(r, t, L[e]);
      }
    } else {
#pragma unroll
      for (int e = 0; e < VN; ++e) {
        const int64_t i = i0 + e;
        const real lc = (i >= 1 && i <= N - 2) ? L[e] : zero;
        const real ll = (i - 1 >= 1 && i - 1 <= N - 2) ? (e > 0 ? L[e - 1] : lleft) : zero;
        const real lr = (i + 1 >= 1 && i + 1 <= N - 2) ? (e + 1 < VN ? L[e + 1] : lright) : zero;
        const real t = adj_lap(one, lc, ll, lr);
        acc = adj_prod(U[e], t, acc);
        if (i == 0 || i == N - 1) {
          out[e] = zero;
          continue;
        }
        real tl = t;  // t without the neighbour terms that arrive delayed
        real pending = 0;
        bool parked = false;
        if (kInline) {
          sg.advance(i, g);
          const int s = sg.s;
          const bool first = s > 0 && i == sg.lo;
          const bool last = s + 1 < g.S && i == sg.hi - 1;
          if (first || last) {
            parked = true;
            double* prow = pend + (k % g.Q) * g.nrods * (g.S - 1) * 2;
            if (first) {
              double* p = prow + (rod * (g.S - 1) + (s - 1)) * 2 + 0;  // parked from i-1's delayed right reads
              pending += static_cast<real>(*p);
              *p = 0.0;
              if (delay_at(g, rod, k, s - 1, 0) > 0) tl -= ll;  // i-1 read u_i late: its term is parked
              const int dL = delay_at(g, rod, k, s - 1, 1);   // this point's own left read
              if (dL > 0) {
                const double uLd = static_cast<double>(eh_row(eh, g, k - dL - t0)[(rod * (g.S - 1) + (s - 1)) * 2 + 1]);
                adj_term(acc, contrib, static_cast<double>(lc) * (uLd - static_cast<double>(ur[i - 1])));
                pend[((k - dL) % g.Q) * g.nrods * (g.S - 1) * 2 + (rod * (g.S - 1) + (s - 1)) * 2 + 1] += r * lc;
              }
            }
            if (last) {
              double* p = prow + (rod * (g.S - 1) + s) * 2 + 1;  // parked from i+1's delayed left reads
              pending += static_cast<real>(*p);
              *p = 0.0;
              if (delay_at(g, rod, k, s, 1) > 0) tl -= lr;    // i+1 read u_i late
              const int dR = delay_at(g, rod, k, s, 0);       // this point's own right read
              if (dR > 0) {
                const double uRd = static_cast<double>(eh_row(eh, g, k - dR - t0)[(rod * (g.S - 1) + s) * 2 + 0]);
                adj_term(acc, contrib, static_cast<double>(lc) * (uRd - static_cast<double>(ur[i + 1])));
                pend[((k - dR) % g.Q) * g.nrods * (g.S - 1) * 2 + (rod * (g.S - 1) + s) * 2 + 0] += r * lc;
              }
            }
          }
        }
        out[e] = parked ? adj_new(one, r, tl, lc, pending) : adj_new0(r, tl, lc);
      }
    }
    V o;
    real* ov = reinterpret_cast<real*>(&o);
#pragma unroll
    for (int e = 0; e < VN; ++e) ov[e] = out[e];
    *reinterpret_cast<V*>(lout + base + i0) = o;
  }
  if (kFix) {  // the block's segment-boundary points, redone with their delayed reads
    __syncthreads();
    bwd_fixup<real>(g, k, lin, lout, ur, eh, t0, pend, rod, base, b0, b1, r, one, acc, contrib);
  }
  const double bs = block_sum_acc<kTrace>(acc, contrib, red);
  if (threadIdx.x == 0) kahan_add(gr_sum + blockIdx.x, gr_comp + blockIdx.x, bs);
}

// lambda(0) of an FP32 run into the caller's FP64 gradient array.
template <typename real>
__global__ void adj_widen(const real* __restrict__ lam, double* __restrict__ out, int64_t n) {
  for (int64_t x = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; x < n;
       x += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[x] = static_cast<double>(lam[x]);
}

// Per rod: sums of the block partials, in block order.
__global__ void adj_finish(AdjGeom g, const double* loss_part, const double* gr_sum, double* loss_out,
                           double* gr_out) {
  const int64_t rod = blockIdx.x * blockDim.x + threadIdx.x;
  if (rod >= g.nrods) return;
  double ls = 0.0, lc = 0.0, gs = 0.0, gc = 0.0;
  for (int64_t b = 0; b < g.bpr; ++b) {
    kahan_add(&ls, &lc, loss_part[rod * g.bpr + b]);
    kahan_add(&gs, &gc, gr_sum[rod * g.bpr + b]);
  }
  loss_out[rod] = ls;
  gr_out[rod] = gs;
}

// One forward step over all rods: the vector kernel where rows are 16-byte aligned.
template <typename real>
void fwd_step(bool vec, dim3 grid, dim3 block, cudaStream_t st, const AdjGeom& g, int64_t k, const real* in,
              real* out, real* eh, int64_t t0) {
  if (vec && g.trace)
    adj_fwd_step_vec<real, true><<<grid, block, 0, st>>>(g, k, in, out, eh, t0);
  else if (vec)
    adj_fwd_step_vec<real, false><<<grid, block, 0, st>>>(g, k, in, out, eh, t0);
  else
    adj_fwd_step<real><<<grid, block, 0, st>>>(g, k, in, out, eh, t0);
}

// One backward step over all rods.
template <typename real>
void bwd_step(bool vec, dim3 grid, dim3 block, cudaStream_t st, const AdjGeom& g, int64_t k, const real* lin,
              real* lout, const real* x, const real* eh, int64_t t0, double* pend, double* gr_sum, double* gr_comp) {
  if (vec && g.trace)
    adj_bwd_step_vec<real, true><<<grid, block, 0, st>>>(g, k, lin, lout, x, eh, t0, pend, gr_sum, gr_comp);
  else if (vec)
    adj_bwd_step_vec<real, false><<<grid, block, 0, st>>>(g, k, lin, lout, x, eh, t0, pend, gr_sum, gr_comp);
  else
    adj_bwd_step<real><<<grid, block, 0, st>>>(g, k, lin, lout, x, eh, t0, pend, gr_sum, gr_comp);
}

template <typename real>
int adjoint_t(const AdjointRun& a) {
  cudaStream_t st = a.stream;
  const int64_t nr = a.nrods, N = a.N, K = a.K, C = std::max<int64_t>(1, std::min<int64_t>(a.ckpt_every, K));
  const int64_t npts = nr * N;
  const bool async_run = a.trace != nullptr;
  const int S = async_run ? a.S : 1;
  const int q = async_run ? a.q : 1;
  AdjGeom g{};
  g.nrods = nr;
  g.N = N;
  g.S = S;
  g.seg_base = N / S;
  g.seg_extra = N % S;
  g.q = q;
  g.Q = q + 1;
  g.span = static_cast<int64_t>(kAdjThreads) * adj_points_per_thread<real>();
  g.bpr = (N + g.span - 1) / g.span;
  g.trace = a.trace;
  g.K = K;
  const int64_t nblocks = nr * g.bpr;
  const int64_t nc = (K + C - 1) / C;  // intervals
  const int64_t ehw = async_run ? nr * (S - 1) * 2 : 0;  // history row width
  const int64_t eh_rows = C + q;                          // times [kc-q+1, kc+C]

  // scratch
  std::vector<void*> owned;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    owned.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    for (void* p : owned) cudaFree(p);
  };
  double* d_coef = static_cast<double*>(alloc(sizeof(double) * 3 * nr));
  float* d_coef32 = static_cast<float*>(alloc(sizeof(float) * 3 * nr));
  real* X = static_cast<real*>(alloc(sizeof(real) * (C + 1) * npts));       // interval workspace
  real* ck = static_cast<real*>(alloc(sizeof(real) * nc * npts));           // checkpoints u(kc)
  real* eh = static_cast<real*>(alloc(sizeof(real) * eh_rows * std::max<int64_t>(ehw, 1)));
  real* ckeh = static_cast<real*>(alloc(sizeof(real) * nc * q * std::max<int64_t>(ehw, 1)));
  real* lam = static_cast<real*>(alloc(sizeof(real) * 2 * npts));
  double* pend = static_cast<double*>(alloc(sizeof(double) * g.Q * std::max<int64_t>(ehw, 1)));
  double* parts = static_cast<double*>(alloc(sizeof(double) * 3 * nblocks));
  double* outs = static_cast<double*>(alloc(sizeof(double) * 2 * nr));
  if (!d_coef || !d_coef32 || !X || !ck || !eh || !ckeh || !lam || !pend || !parts || !outs) {
    cleanup();
    return HEAT1D_ERR_OOM;
  }
  std::vector<double> coef(3 * nr);
  for (int64_t j = 0; j < nr; ++j) {
    coef[j] = a.r[j];
    coef[nr + j] = a.c1[j];
    coef[2 * nr + j] = a.cN[j];
  }
  std::vector<float> coef32(coef.begin(), coef.end());
  g.r = d_coef;
  g.c1 = d_coef + nr;
  g.cN = d_coef + 2 * nr;
  g.rf = d_coef32;
  g.c1f = d_coef32 + nr;
  g.cNf = d_coef32 + 2 * nr;
  cudaError_t e = cudaMemcpyAsync(d_coef, coef.data(), sizeof(double) * 3 * nr, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_coef32, coef32.data(), sizeof(float) * 3 * nr, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pend, 0, sizeof(double) * g.Q * std::max<int64_t>(ehw, 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(parts, 0, sizeof(double) * 3 * nblocks, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(X, a.u0, sizeof(real) * npts, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    cleanup();
    return HEAT1D_ERR_CUDA;
  }
  const dim3 grid(static_cast<unsigned>(nblocks)), block(kAdjThreads);
  // 16-byte vectors where every rod row starts on a 16-byte boundary (the
  // blocks' span, kAdjThreads * adj_points_per_thread, is a multiple of the
  // vector width times kAdjThreads)
  const bool vec = N % Vec16T<real>::n == 0 && g.span % (static_cast<int64_t>(kAdjThreads) * Vec16T<real>::n) == 0;
  const bool bvec = vec;
  const int gather_blocks = static_cast<int>(std::min<int64_t>(1024, (std::max<int64_t>(ehw / 2, 1) + 255) / 256));
  adj_force_ends<real><<<static_cast<unsigned>((nr + 127) / 128), 128, 0, st>>>(g, X);  // u(0) with its ends set
  // history rows for times <= 0 all hold u(0) (reads before 0 are clamped, so
  // only the row of time 0 is ever read)
  if (async_run) {
    for (int64_t row = 0; row < q; ++row)
      adj_edge_gather<real><<<gather_blocks, 256, 0, st>>>(g, X, eh + row * ehw);
  }

  // ---- forward with checkpoints
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t kc = c * C, Cc = std::min<int64_t>(C, K - kc);
    const int64_t t0 = kc - (q - 1);
    if (c > 0) {  // the interval starts from the previous interval's last state and history
      e = cudaMemcpyAsync(X, X + C * npts, sizeof(real) * npts, cudaMemcpyDeviceToDevice, st);
      if (e == cudaSuccess && async_run)
        e = cudaMemcpyAsync(eh, eh + C * ehw, sizeof(real) * q * ehw, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) break;
    }
    e = cudaMemcpyAsync(ck + c * npts, X, sizeof(real) * npts, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && async_run)
      e = cudaMemcpyAsync(ckeh + c * q * ehw, eh, sizeof(real) * q * ehw, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) break;
    for (int64_t j = 0; j < Cc; ++j)
      fwd_step<real>(vec, grid, block, st, g, kc + j, X + j * npts, X + (j + 1) * npts, eh, t0);
    if (c == nc - 1 && Cc != C)  // make the final state sit where the next interval would look
      e = cudaMemcpyAsync(X + C * npts, X + Cc * npts, sizeof(real) * npts, cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && a.uK)
    e = cudaMemcpyAsync(a.uK, X + C * npts, sizeof(real) * npts, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    cleanup();
    return HEAT1D_ERR_CUDA;
  }
  real* lin = lam;
  real* lout = lam + npts;
  adj_init<real><<<grid, block, 0, st>>>(g, X + C * npts, a.u_obs, lin, parts, a.cotangent);

  // ---- backward: recompute each interval, then march lambda back through it
  for (int64_t c = nc - 1; c >= 0 && e == cudaSuccess; --c) {
    const int64_t kc = c * C, Cc = std::min<int64_t>(C, K - kc);
    const int64_t t0 = kc - (q - 1);
    e = cudaMemcpyAsync(X, ck + c * npts, sizeof(real) * npts, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && async_run)
      e = cudaMemcpyAsync(eh, ckeh + c * q * ehw, sizeof(real) * q * ehw, cudaMemcpyDeviceToDevice, st);
    for (int64_t j = 0; j + 1 < Cc && e == cudaSuccess; ++j)  // states kc .. kc+Cc-1
      fwd_step<real>(vec, grid, block, st, g, kc + j, X + j * npts, X + (j + 1) * npts, eh, t0);
    for (int64_t k = kc + Cc - 1; k >= kc; --k) {
      bwd_step<real>(bvec, grid, block, st, g, k, lin, lout, X + (k - kc) * npts, eh, t0, pend, parts + nblocks,
                     parts + 2 * nblocks);
      std::swap(lin, lout);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    adj_finish<<<static_cast<unsigned>((nr + 127) / 128), 128, 0, st>>>(g, parts, parts + nblocks, outs, outs + nr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    if (sizeof(real) == sizeof(double)) {
      e = cudaMemcpyAsync(a.grad_u0, lin, sizeof(double) * npts, cudaMemcpyDeviceToDevice, st);
    } else {
      adj_widen<real><<<static_cast<unsigned>(std::min<int64_t>((npts + 255) / 256, 65535)), 256, 0, st>>>(
          lin, a.grad_u0, npts);
      e = cudaGetLastError();
    }
  }
  std::vector<double> host(2 * nr);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), outs, sizeof(double) * 2 * nr, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return HEAT1D_ERR_CUDA;
  for (int64_t j = 0; j < nr; ++j) {
    if (a.loss) a.loss[j] = host[j];
    if (a.grad_r) a.grad_r[j] = host[nr + j];
  }
  return HEAT1D_OK;
}

}  // namespace

int run_adjoint(const AdjointRun& a, int dtype) {
  return dtype == HEAT1D_F64 ? adjoint_t<double>(a) : adjoint_t<float>(a);
}

}  // namespace heat1d_impl

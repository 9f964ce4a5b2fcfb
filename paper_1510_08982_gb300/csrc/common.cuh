// common.cuh -- device helpers shared by the heat1d kernels (sm_103a).
//
// Memory-model helpers (PTX release/acquire at gpu and cta scope), the
// bounded-wait clock, the status word, and the register-tile FTCS step that
// every kernel of the library is built from.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "heat1d.h"
#include "impl.h"

namespace heat1d_dev {

constexpr unsigned kFullMask = 0xffffffffu;

// ------------------------------------------------------------ memory model

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_gpu(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Shared-memory flags between warps of one CTA.
__device__ __forceinline__ int ld_acquire_cta_shared(const int* p) {
  int v;
  unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_cta_shared(int* p, int v) {
  unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Values crossing CTAs: read at L2 (never a stale L1 line), written through.
template <typename real>
__device__ __forceinline__ real ld_cg(const real* p) { return __ldcg(p); }
template <typename real>
__device__ __forceinline__ void st_cg(real* p, real v) { __stcg(p, v); }

// Named barrier over `nthreads` threads of the CTA (id 1; id 0 is
// __syncthreads).  Lets a communication warp stay out of the compute warps'
// step barrier.  The non-.aligned form is used: it stays correct even if the
// compiler does not reconverge a warp before the barrier.
__device__ __forceinline__ void named_barrier_sync(unsigned id, unsigned nthreads) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Same barrier, returning the OR of `pred` over the participating threads.
__device__ __forceinline__ bool named_barrier_or(unsigned id, unsigned nthreads, bool pred) {
  int out;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.s32 pi, %1, 0;\n\t"
      "barrier.red.or.pred po, %2, %3, pi;\n\t"
      "selp.s32 %0, 1, 0, po;\n\t}"
      : "=r"(out)
      : "r"((int)pred), "r"(id), "r"(nthreads)
      : "memory");
  return out != 0;
}

// ------------------------------------------------------------ status word

// Device status: 0 while healthy; the first failure stores its (negative)
// heat1d_status code and every bounded wait in every CTA then gives up.
__device__ __forceinline__ void raise_status(int* status, int code) { atomicCAS(status, 0, code); }
__device__ __forceinline__ bool status_failed(const int* status) { return ld_relaxed_gpu(status) != 0; }

// ------------------------------------------------------------ FTCS arithmetic

// One interior update in the order of the paper's printed kernels
// (Section 4): r*(uR - 2u + uL) + u with the final multiply-add fused.
// uR - 2u is formed by one fused multiply-add, which equals the rounded
// difference because 2u is exact.  Explicit _rn intrinsics forbid any other
// contraction, so the result is the same, bit for bit, as the CPU oracle's.
//
// In FP64 the middle addition is also issued as a fused multiply-add,
// fma(one, t, uL) with one == 1.0: the product is exact, so the result is the
// rounded sum, bit for bit.  On GB300 the FP64 pipe sustains DFMA at a higher
// rate than DADD (measured 5.96e11/s against 5.02e11/s), and an update then
// costs three DFMA.  `one` is a run-time value so that the compiler cannot
// turn the FMA back into an add.
__device__ __forceinline__ double ftcs(double r, double one, double uL, double u, double uR) {
  return __fma_rn(r, __fma_rn(one, __fma_rn(-2.0, u, uR), uL), u);
}
__device__ __forceinline__ float ftcs(float r, float /*one*/, float uL, float u, float uR) {
  return __fmaf_rn(r, __fadd_rn(__fmaf_rn(-2.0f, u, uR), uL), u);
}

// ------------------------------------------------------------ warp windows
//
// The compute warps of a CTA hold a contiguous run of points ("positions")
// in registers.  Warp w covers the window of 32*E positions starting at w*D,
// D = 32*E - 2*H, 1 <= H <= E/2: lane l holds positions w*D + l*E + e in v[e].
// Adjacent windows overlap by 2*H positions, so each warp carries H halo
// points on each side that belong to its neighbours.
//
// A step inside a warp needs no other warp: neighbours within a thread come
// from registers, across lanes from shuffles; lane 0's first point and lane
// 31's last point read garbage and become invalid, and the invalid region
// grows by one point per side per step.  After at most H steps the warps
// refresh their halos from their neighbours' valid points through shared
// memory, with one CTA barrier.  The redundant work is 2H/(32E) of the
// arithmetic and the warps synchronise once per H steps, not per step
// (the choice of H per kernel is in impl.h).
// Because the halo points are recomputed with the same arithmetic, results
// are bit-identical to updating every point once per step.
//
// Positions whose bit in `fixed` is set keep their value (Dirichlet ends,
// halo points written from outside, padding).  Positions in an overlap are
// held by two warps; only the "owner" (warp w owns its interior positions
// [w*D + H, w*D + 32E - H); warp 0 and the last warp also own the CTA's outer
// H positions) publishes or stores them.

// A run parameter in the run's precision: F64 kernels take the double, F32
// kernels the float the host rounded it to.  The kernels then never convert a
// double to float, which runs on the FP64 pipe and which the compiler may
// repeat wherever it recomputes the value instead of keeping it in a
// register (measured: one conversion per warp and halo refresh in the FP32
// synchronous kernel).
template <typename real>
__device__ __forceinline__ real kparam(double d, float f);
template <>
__device__ __forceinline__ double kparam<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float kparam<float>(double, float f) { return f; }

// Stencil coefficients: r, and a run-time 1.0 (see ftcs).
template <typename real>
struct Coef {
  real r;
  real one;
};

template <int E, int H_>
struct Window {
  static_assert(E >= 2 && E % 2 == 0, "E must be even");
  static constexpr int H = H_;            // halo points per warp side
  static constexpr int D = 32 * E - 2 * H;  // stride between warp windows
  // Either half a lane (the halos and the values sent for them sit in lanes
  // 0 and 31) or a whole lane (H = E: lanes 0 and 31 are the halos, lanes 1
  // and 30 send).
  static_assert(H >= 1 && (2 * H <= E || H == E), "halo must be at most half a lane, or one whole lane");
  __device__ static __forceinline__ int pos(int warp, int lane, int e) { return warp * D + lane * E + e; }
  // Whether the warp's window holds any of the positions [a, b): a test that
  // is the same for every lane, so that the warps holding none of an edge
  // strip skip the per-point loop that reads or writes it.
  __device__ static __forceinline__ bool touches(int warp, int a, int b) {
    return warp * D < b && warp * D + 32 * E > a;
  }
  __device__ static __forceinline__ bool owner(int warp, int lane, int e, int nwarps) {
    if (lane == 0 && e < H) return warp == 0;
    if (lane == 31 && e >= E - H) return warp == nwarps - 1;
    return true;
  }
};

// Halo exchange buffers: two parities (a warp cannot write parity p again
// before every warp passed the barrier of the refresh in between).
template <typename real, int H>
struct WindowShared {
  real to_right[2][32][H];  // window positions [32E-2H, 32E-H): the next warp's left halo
  real to_left[2][32][H];   // window positions [H, 2H): the previous warp's right halo
};

// How a warp steps: every point updated; the first and/or last slot of some
// lanes held (a Dirichlet end placed at a slot known at compile time: two
// selects per step); any other points held (a select per point); or every
// point held (padding warps: no arithmetic).  kTileSlot + s (1 <= s <= E-2):
// slot 0 and slot s of some lanes held -- a rod's first point and its last
// point u_N, which falls at slot (N-1) mod E -- as a mode of its own for
// every s, so that the two holds cost two selects per step instead of one
// per point (measured: a warp in the per-point mode slows its whole CTA by a
// quarter, as every warp waits for it at each refresh).
enum TileMode { kTileFree = 0, kTileMasked = 1, kTileIdle = 2, kTileEnds = 3, kTileSlot = 4 };

// Whether slot e may be held in mode kMode (then its `fixed` bit decides).
template <int E, int kMode>
__device__ __forceinline__ constexpr bool held_slot(int e) {
  return kMode == kTileMasked || (kMode == kTileEnds && (e == 0 || e == E - 1)) ||
         (kMode >= kTileSlot && (e == 0 || e == kMode - kTileSlot));
}

// Kernels hold only the Dirichlet ends: positions outside the rod or past the
// tile are stepped like any other (their values are never stored and reach no
// stored point before they are overwritten or the tile ends), so that no warp
// pays per-point selects for padding.
template <int E>
__device__ __forceinline__ int tile_mode(unsigned fixed) {
  const unsigned all = (E >= 32) ? 0xffffffffu : ((1u << E) - 1u);
  if (__all_sync(kFullMask, fixed == all)) return kTileIdle;
  if (!__any_sync(kFullMask, fixed != 0u)) return kTileFree;
  const unsigned ends = 1u | (1u << (E - 1));
  return __any_sync(kFullMask, (fixed & ~ends) != 0u) ? kTileMasked : kTileEnds;
}

// tile_mode, with the slot modes: a warp whose held points are at slot 0 and
// at one other slot s (the same in every lane) steps in mode kTileSlot + s.
// Only for E <= 16 (the number of step-loop copies grows with E).
template <int E>
__device__ __forceinline__ int tile_mode_slot(unsigned fixed) {
  const int mode = tile_mode<E>(fixed);
  if (E > 16 || mode != kTileMasked) return mode;
  const unsigned inner = __reduce_or_sync(kFullMask, fixed) & ~1u;
  if ((inner & (inner - 1u)) != 0u) return kTileMasked;  // two inner slots
  const int s = __ffs(static_cast<int>(inner)) - 1;
  return (s >= 1 && s <= E - 2) ? kTileSlot + s : kTileMasked;
}

// One step of one warp (no other warp involved).
template <typename real, int E, int kMode>
__device__ __forceinline__ void warp_step(real (&v)[E], unsigned fixed, Coef<real> c) {
  const real left = __shfl_up_sync(kFullMask, v[E - 1], 1);
  const real right = __shfl_down_sync(kFullMask, v[0], 1);
  if (kMode == kTileIdle) return;
  real prev = left;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const real cur = v[e];
    const real nxt = (e + 1 < E) ? v[e + 1] : right;
    const real nv = ftcs(c.r, c.one, prev, cur, nxt);
    if (held_slot<E, kMode>(e)) {
      v[e] = ((fixed >> e) & 1u) ? cur : nv;
    } else {
      v[e] = nv;
    }
    prev = cur;
  }
}

// The same step from `in` to `out` (separate registers).
template <typename real, int E, int kMode>
__device__ __forceinline__ void warp_step_to(const real (&in)[E], real (&out)[E], unsigned fixed, Coef<real> c) {
  const real left = __shfl_up_sync(kFullMask, in[E - 1], 1);
  const real right = __shfl_down_sync(kFullMask, in[0], 1);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const real prev = e > 0 ? in[e - 1] : left;
    const real nxt = (e + 1 < E) ? in[e + 1] : right;
    const real nv = ftcs(c.r, c.one, prev, in[e], nxt);
    if (held_slot<E, kMode>(e)) {
      out[e] = ((fixed >> e) & 1u) ? in[e] : nv;
    } else {
      out[e] = nv;
    }
  }
}

// n steps of one warp, two at a time between two register arrays, so that
// the loop carries no register moves.
template <typename real, int E, int kMode>
__device__ __forceinline__ void warp_steps(real (&v)[E], unsigned fixed, Coef<real> c, int64_t n) {
  if (kMode == kTileIdle) {
    for (int64_t j = 0; j < n; ++j) warp_step<real, E, kTileIdle>(v, fixed, c);
    return;
  }
  real w[E];
  int64_t j = 0;
  for (; j + 1 < n; j += 2) {
    warp_step_to<real, E, kMode>(v, w, fixed, c);
    warp_step_to<real, E, kMode>(w, v, fixed, c);
  }
  if (j < n) warp_step<real, E, kMode>(v, fixed, c);
}

// A run of n <= H steps between two halo refreshes.  A full run of H steps
// (the common case) is unrolled completely, so that no step pays a loop
// counter, a compare or a branch; a shorter run takes the loop.
template <typename real, int E, int kMode, int H>
__device__ __forceinline__ void warp_run(real (&v)[E], unsigned fixed, Coef<real> c, int n) {
  if (kMode == kTileIdle) return;  // a warp wholly outside the tile holds nothing that is read
  if (n != H) {
    warp_steps<real, E, kMode>(v, fixed, c, n);
    return;
  }
  real w[E];
#pragma unroll
  for (int j = 0; j + 1 < H; j += 2) {
    warp_step_to<real, E, kMode>(v, w, fixed, c);
    warp_step_to<real, E, kMode>(w, v, fixed, c);
  }
  if (H & 1) warp_step<real, E, kMode>(v, fixed, c);
}

template <typename real, int E>
__device__ __forceinline__ void warp_step_any(int mode, real (&v)[E], unsigned fixed, Coef<real> c) {
  if (mode == kTileFree)
    warp_step<real, E, kTileFree>(v, fixed, c);
  else if (mode == kTileEnds)
    warp_step<real, E, kTileEnds>(v, fixed, c);
  else if (mode == kTileMasked)
    warp_step<real, E, kTileMasked>(v, fixed, c);
  else
    warp_step<real, E, kTileIdle>(v, fixed, c);
}

// Refreshes every warp's halos from its neighbours (one barrier over the
// `nthreads` compute threads, named barrier 1).  kOr: the barrier also
// returns the OR of `flag` over those threads, so that a failure seen by one
// thread reaches all of them at the same point; otherwise a plain barrier.
template <typename real, int E, int H, bool kOr = true>
__device__ __forceinline__ bool warp_refresh(real (&v)[E], WindowShared<real, H>& sh, int parity, int warp, int lane,
                                             int nwarps, unsigned nthreads, bool flag) {
  // The next warp's left halo is this warp's window positions [32E-2H,
  // 32E-H); the previous warp's right halo is positions [H, 2H).  With
  // H <= E/2 those are in lanes 31 and 0, with H = E they are lanes 30 and 1.
  constexpr bool kLane = (H == E);
  if (lane == (kLane ? 30 : 31)) {
#pragma unroll
    for (int i = 0; i < H; ++i) sh.to_right[parity][warp][i] = v[kLane ? i : E - 2 * H + i];
  }
  if (lane == (kLane ? 1 : 0)) {
#pragma unroll
    for (int i = 0; i < H; ++i) sh.to_left[parity][warp][i] = v[kLane ? i : H + i];
  }
  bool any = false;
  if (kOr)
    any = named_barrier_or(1, nthreads, flag);
  else
    named_barrier_sync(1, nthreads);
  if (lane == 0 && warp > 0) {
#pragma unroll
    for (int i = 0; i < H; ++i) v[i] = sh.to_right[parity][warp - 1][i];
  }
  if (lane == 31 && warp + 1 < nwarps) {
#pragma unroll
    for (int i = 0; i < H; ++i) v[E - H + i] = sh.to_left[parity][warp + 1][i];
  }
  return any;
}

// warp_advance for one tile mode: full runs of H steps (unrolled), each
// followed by a refresh, then the last run of 1..H steps.
template <typename real, int E, int H, int kMode>
__device__ __forceinline__ void warp_advance_mode(real (&v)[E], unsigned fixed, Coef<real> c,
                                                  WindowShared<real, H>& sh, int& parity, int warp, int lane,
                                                  int nwarps, unsigned nthreads, int steps, bool final_refresh) {
  int done = 0;
  for (; done + H < steps; done += H) {
    warp_run<real, E, kMode, H>(v, fixed, c, H);
    warp_refresh<real, E, H, false>(v, sh, parity, warp, lane, nwarps, nthreads, false);
    parity ^= 1;
  }
  warp_run<real, E, kMode, H>(v, fixed, c, steps - done);
  if (final_refresh) {
    warp_refresh<real, E, H, false>(v, sh, parity, warp, lane, nwarps, nthreads, false);
    parity ^= 1;
  }
}

// Advances the CTA `steps` steps: runs of at most H warp steps, each followed
// by a refresh, so the windows are fully valid again when it returns.  With
// final_refresh = false the refresh after the last run is left out: every
// warp's own positions are valid after at most H steps, and a caller that
// only stores those (and then discards the tile) saves a barrier; with
// steps <= H no barrier is met at all.  The mode is resolved once per call.
template <typename real, int E, int H>
__device__ __forceinline__ void warp_advance(int mode, real (&v)[E], unsigned fixed, Coef<real> c,
                                             WindowShared<real, H>& sh, int& parity, int warp, int lane, int nwarps,
                                             unsigned nthreads, int steps, bool final_refresh = true) {
  if (steps <= 0) return;
  if (mode == kTileFree)
    warp_advance_mode<real, E, H, kTileFree>(v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps,
                                             final_refresh);
  else if (mode == kTileEnds)
    warp_advance_mode<real, E, H, kTileEnds>(v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps,
                                             final_refresh);
  else if (mode == kTileMasked)
    warp_advance_mode<real, E, H, kTileMasked>(v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps,
                                               final_refresh);
  else
    warp_advance_mode<real, E, H, kTileIdle>(v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps,
                                             final_refresh);
}

// warp_advance with the slot modes of tile_mode_slot (one copy of the step
// loop per slot, chosen once per call).
template <typename real, int E, int H, int S = 1>
__device__ __forceinline__ void warp_advance_slot(int s, real (&v)[E], unsigned fixed, Coef<real> c,
                                                  WindowShared<real, H>& sh, int& parity, int warp, int lane,
                                                  int nwarps, unsigned nthreads, int steps, bool final_refresh) {
  if constexpr (S <= E - 2) {
    if (s == S)
      warp_advance_mode<real, E, H, kTileSlot + S>(v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps,
                                                   final_refresh);
    else
      warp_advance_slot<real, E, H, S + 1>(s, v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps,
                                           final_refresh);
  }
}
template <typename real, int E, int H>
__device__ __forceinline__ void warp_advance_slots(int mode, real (&v)[E], unsigned fixed, Coef<real> c,
                                                   WindowShared<real, H>& sh, int& parity, int warp, int lane,
                                                   int nwarps, unsigned nthreads, int steps,
                                                   bool final_refresh = true) {
  if (steps <= 0) return;
  if (mode >= kTileSlot)
    warp_advance_slot<real, E, H>(mode - kTileSlot, v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps,
                                  final_refresh);
  else
    warp_advance<real, E, H>(mode, v, fixed, c, sh, parity, warp, lane, nwarps, nthreads, steps, final_refresh);
}

// warp_steps with the slot modes (a warp that holds a whole rod).
template <typename real, int E, int S = 1>
__device__ __forceinline__ void warp_steps_slot(int s, real (&v)[E], unsigned fixed, Coef<real> c, int64_t n) {
  if constexpr (S <= E - 2) {
    if (s == S)
      warp_steps<real, E, kTileSlot + S>(v, fixed, c, n);
    else
      warp_steps_slot<real, E, S + 1>(s, v, fixed, c, n);
  }
}

__device__ __forceinline__ int ld_volatile_shared(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

}  // namespace heat1d_dev

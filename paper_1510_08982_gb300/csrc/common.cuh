// common.cuh -- device helpers shared by the heat1d kernels (sm_103a).
//
// Memory-model helpers (PTX release/acquire at gpu and cta scope), the
// bounded-wait clock, the status word, and the register-tile FTCS step that
// every kernel of the library is built from.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "heat1d.h"

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

// ------------------------------------------------------------ register tile
//
// A CTA (or its compute warps) holds a contiguous run of "slots" in registers:
// thread t holds slots t*E .. t*E+E-1 in v[0..E-1].  One step updates every
// slot whose bit in `fixed` is clear from its two neighbours; neighbours in
// the same thread come from registers, across lanes from shuffles, and across
// warps from shared memory.  Slots whose bit is set keep their value
// (Dirichlet ends, halo ends, padding).
//
// There is no CTA-wide barrier per step.  Lane 0 and lane 31 of warp w publish
// the warp's first and last value of step k in a two-parity shared array and
// then a per-warp flag (release at CTA scope); lane 0 of warp w+1 and lane 31
// of warp w-1 wait for that flag (acquire) before reading.  A warp therefore
// waits only for its two neighbours, and warps may be one step apart, which
// keeps the arithmetic pipe busy across step boundaries.  Two parities
// suffice: a warp cannot publish step k+2 (overwriting step k) before both
// neighbours have published step k+1, i.e. have finished reading step k.

template <typename real>
struct TileShared {
  real first[2][32];      // v[0] of lane 0 of each warp, per step parity
  real last[2][32];       // v[E-1] of lane 31 of each warp, per step parity
  unsigned fflag[32];     // step whose `first` value warp w has published (+1; 0 = none)
  unsigned lflag[32];     // same for `last`
  int abort;              // non-zero: stop waiting, leave the step loop
};

// Must be called by the CTA before the first step, followed by a barrier.
template <typename real>
__device__ __forceinline__ void tile_shared_init(TileShared<real>& sh, int tid) {
  if (tid < 32) {
    sh.fflag[tid] = 0u;
    sh.lflag[tid] = 0u;
  }
  if (tid == 0) sh.abort = 0;
}

__device__ __forceinline__ unsigned ld_acquire_cta_shared_u32(const unsigned* p) {
  unsigned v;
  unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_cta_shared_u32(unsigned* p, unsigned v) {
  unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(p));
  asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_shared(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Waits until *flag has reached `want` (wrap-safe).  Gives up, setting the
// CTA's abort flag, when the abort flag is already set or after `limit_ns`.
static __device__ __noinline__ bool tile_wait_flag(const unsigned* flag, unsigned want, int* abort, int64_t limit_ns) {
  unsigned spins = 0;
  uint64_t t0 = 0;
  while (static_cast<int>(ld_acquire_cta_shared_u32(flag) - want) < 0) {
    if (ld_volatile_shared(abort)) return false;
    if ((++spins & 255u) == 0) {
      const uint64_t t = global_timer_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (static_cast<int64_t>(t - t0) > limit_ns) {
        *reinterpret_cast<volatile int*>(abort) = 1;
        return false;
      }
    }
  }
  return true;
}

// Stencil coefficients: r, and a run-time 1.0 (see ftcs).
template <typename real>
struct Coef {
  real r;
  real one;
};

// How a warp steps: every slot updated, some slots fixed (select), or every
// slot fixed (padding warps: no arithmetic, but they publish and wait like the
// others, so that no warp runs ahead of its neighbours -- a halo slot written
// from outside the tile may sit in such a warp).
enum TileMode { kTileFree = 0, kTileMasked = 1, kTileIdle = 2 };

template <int E>
__device__ __forceinline__ int tile_mode(unsigned fixed) {
  const unsigned all = (E >= 32) ? 0xffffffffu : ((1u << E) - 1u);
  if (__all_sync(kFullMask, fixed == all)) return kTileIdle;
  return __any_sync(kFullMask, fixed != 0u) ? kTileMasked : kTileFree;
}

// One step k -> k+1 of the warp.  Returns false (warp-uniform) if a wait gave
// up because the CTA is aborting; the values are then unspecified.
template <typename real, int E, int kMode>
__device__ __forceinline__ bool tile_step(real (&v)[E], unsigned fixed, Coef<real> c, TileShared<real>& sh,
                                          unsigned k, int warp, int lane, int nwarps, int64_t limit_ns) {
  const int p = k & 1u;
  if (lane == 0) {
    sh.first[p][warp] = v[0];
    st_release_cta_shared_u32(&sh.fflag[warp], k + 1u);
  }
  if (lane == 31) {
    sh.last[p][warp] = v[E - 1];
    st_release_cta_shared_u32(&sh.lflag[warp], k + 1u);
  }
  real left = __shfl_up_sync(kFullMask, v[E - 1], 1);
  real right = __shfl_down_sync(kFullMask, v[0], 1);
  bool ok = true;
  if (lane == 0 && warp > 0) {
    ok = tile_wait_flag(&sh.lflag[warp - 1], k + 1u, &sh.abort, limit_ns);
    left = sh.last[p][warp - 1];
  }
  if (lane == 31 && warp + 1 < nwarps) {
    ok = tile_wait_flag(&sh.fflag[warp + 1], k + 1u, &sh.abort, limit_ns);
    right = sh.first[p][warp + 1];
  }
  if (!__all_sync(kFullMask, ok)) return false;
  if (kMode == kTileIdle) return true;
  real prev = left;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const real cur = v[e];
    const real nxt = (e + 1 < E) ? v[e + 1] : right;
    const real nv = ftcs(c.r, c.one, prev, cur, nxt);
    if (kMode == kTileMasked) {
      v[e] = ((fixed >> e) & 1u) ? cur : nv;
    } else {
      v[e] = nv;
    }
    prev = cur;
  }
  return true;
}

// One step in the warp's mode (mode from tile_mode, warp-uniform).
template <typename real, int E>
__device__ __forceinline__ bool tile_step_any(int mode, real (&v)[E], unsigned fixed, Coef<real> c,
                                              TileShared<real>& sh, unsigned k, int warp, int lane, int nwarps,
                                              int64_t limit_ns) {
  if (mode == kTileFree)
    return tile_step<real, E, kTileFree>(v, fixed, c, sh, k, warp, lane, nwarps, limit_ns);
  if (mode == kTileMasked)
    return tile_step<real, E, kTileMasked>(v, fixed, c, sh, k, warp, lane, nwarps, limit_ns);
  return tile_step<real, E, kTileIdle>(v, fixed, c, sh, k, warp, lane, nwarps, limit_ns);
}

// ------------------------------------------------------------ lockstep tile
//
// The same step with a CTA-wide barrier per step instead of neighbour flags,
// so that no warp is ever more than one step away from any other.  The
// asynchronous run uses it: there the two edge warps must not lag behind the
// rest of the segment, or the delay seen by the neighbouring segments grows
// (with neighbour flags alone the skew across a CTA can reach one step per
// warp).  Two parities of edge values and one barrier per step suffice.

template <typename real>
struct LockstepShared {
  real first[2][32];
  real last[2][32];
  int abort;  // set by a failed wait; every warp leaves at the next step
};

template <typename real, int E, int kMode>
__device__ __forceinline__ void lockstep_step(real (&v)[E], unsigned fixed, Coef<real> c, LockstepShared<real>& sh,
                                              unsigned k, int warp, int lane, int nwarps) {
  const int p = k & 1u;
  if (lane == 0) sh.first[p][warp] = v[0];
  if (lane == 31) sh.last[p][warp] = v[E - 1];
  real left = __shfl_up_sync(kFullMask, v[E - 1], 1);
  real right = __shfl_down_sync(kFullMask, v[0], 1);
  named_barrier_sync(1, static_cast<unsigned>(nwarps) * 32u);
  if (kMode == kTileIdle) return;
  if (lane == 0 && warp > 0) left = sh.last[p][warp - 1];
  if (lane == 31 && warp + 1 < nwarps) right = sh.first[p][warp + 1];
  real prev = left;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const real cur = v[e];
    const real nxt = (e + 1 < E) ? v[e + 1] : right;
    const real nv = ftcs(c.r, c.one, prev, cur, nxt);
    if (kMode == kTileMasked) {
      v[e] = ((fixed >> e) & 1u) ? cur : nv;
    } else {
      v[e] = nv;
    }
    prev = cur;
  }
}

template <typename real, int E>
__device__ __forceinline__ void lockstep_step_any(int mode, real (&v)[E], unsigned fixed, Coef<real> c,
                                                  LockstepShared<real>& sh, unsigned k, int warp, int lane,
                                                  int nwarps) {
  if (mode == kTileFree)
    lockstep_step<real, E, kTileFree>(v, fixed, c, sh, k, warp, lane, nwarps);
  else if (mode == kTileMasked)
    lockstep_step<real, E, kTileMasked>(v, fixed, c, sh, k, warp, lane, nwarps);
  else
    lockstep_step<real, E, kTileIdle>(v, fixed, c, sh, k, warp, lane, nwarps);
}

// Runs steps k0 .. k0+steps-1.  Returns false if the CTA aborted.
template <typename real, int E>
__device__ __forceinline__ bool tile_steps(int mode, real (&v)[E], unsigned fixed, Coef<real> c,
                                           TileShared<real>& sh, unsigned k0, int warp, int lane, int nwarps,
                                           int steps, int64_t limit_ns) {
  bool ok = true;
  if (mode == kTileFree) {
    for (int j = 0; j < steps && ok; ++j)
      ok = tile_step<real, E, kTileFree>(v, fixed, c, sh, k0 + j, warp, lane, nwarps, limit_ns);
  } else if (mode == kTileMasked) {
    for (int j = 0; j < steps && ok; ++j)
      ok = tile_step<real, E, kTileMasked>(v, fixed, c, sh, k0 + j, warp, lane, nwarps, limit_ns);
  } else {
    for (int j = 0; j < steps && ok; ++j)
      ok = tile_step<real, E, kTileIdle>(v, fixed, c, sh, k0 + j, warp, lane, nwarps, limit_ns);
  }
  return ok;
}

}  // namespace heat1d_dev

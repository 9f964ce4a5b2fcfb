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
__device__ __forceinline__ double ftcs(double r, double uL, double u, double uR) {
  return __fma_rn(r, __dadd_rn(__fma_rn(-2.0, u, uR), uL), u);
}
__device__ __forceinline__ float ftcs(float r, float uL, float u, float uR) {
  return __fmaf_rn(r, __fadd_rn(__fmaf_rn(-2.0f, u, uR), uL), u);
}

// ------------------------------------------------------------ register tile
//
// A CTA (or its compute warps) holds a contiguous run of "slots" in registers:
// thread t holds slots t*E .. t*E+E-1 in v[0..E-1].  One step updates every
// slot whose bit in `fixed` is clear from its two neighbours; neighbours in
// the same thread come from registers, across lanes from shuffles, across
// warps from a small shared array (two parities, one barrier per step).
// Slots whose bit is set keep their value (Dirichlet ends, halo ends, padding).

template <typename real>
struct TileShared {
  real first[2][32];  // v[0] of lane 0 of each warp, per parity
  real last[2][32];   // v[E-1] of lane 31 of each warp, per parity
};

template <typename real, int E, bool kHasFixed>
__device__ __forceinline__ bool tile_step(real (&v)[E], unsigned fixed, real r, TileShared<real>& sh, int parity,
                                          int warp, int lane, int nwarps, unsigned barrier_threads, bool flag) {
  if (lane == 0) sh.first[parity][warp] = v[0];
  if (lane == 31) sh.last[parity][warp] = v[E - 1];
  real left = __shfl_up_sync(kFullMask, v[E - 1], 1);
  real right = __shfl_down_sync(kFullMask, v[0], 1);
  const bool any_flag = named_barrier_or(1, barrier_threads, flag);
  if (lane == 0 && warp > 0) left = sh.last[parity][warp - 1];
  if (lane == 31 && warp + 1 < nwarps) right = sh.first[parity][warp + 1];
  real prev = left;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const real cur = v[e];
    const real nxt = (e + 1 < E) ? v[e + 1] : right;
    const real nv = ftcs(r, prev, cur, nxt);
    if (kHasFixed) {
      v[e] = ((fixed >> e) & 1u) ? cur : nv;
    } else {
      v[e] = nv;
    }
    prev = cur;
  }
  return any_flag;
}

// Runs `steps` tile steps with no flag; warps with no fixed slot take the
// select-free path (the choice is warp-uniform so that shuffles and barriers
// stay converged).
template <typename real, int E>
__device__ __forceinline__ void tile_steps(real (&v)[E], unsigned fixed, real r, TileShared<real>& sh, int& parity,
                                           int warp, int lane, int nwarps, unsigned barrier_threads, int steps) {
  if (__any_sync(kFullMask, fixed != 0u)) {
    for (int j = 0; j < steps; ++j) {
      tile_step<real, E, true>(v, fixed, r, sh, parity, warp, lane, nwarps, barrier_threads, false);
      parity ^= 1;
    }
  } else {
    for (int j = 0; j < steps; ++j) {
      tile_step<real, E, false>(v, fixed, r, sh, parity, warp, lane, nwarps, barrier_threads, false);
      parity ^= 1;
    }
  }
}

}  // namespace heat1d_dev

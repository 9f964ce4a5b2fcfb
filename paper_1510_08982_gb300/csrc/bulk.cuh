// bulk.cuh -- shared-memory pipelines fed by bulk copies (sm_103a).
//
// mbarrier helpers (init, arrive, arrive with an expected byte count, a
// bounded wait on a phase) and the 1D bulk copy from global to shared memory
// (cp.async.bulk, the 1D form of TMA) whose completion lands on an mbarrier.
// Used by the streamed kernels: a loader thread copies tiles into a ring of
// shared-memory stages, the compute warps consume them.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace heat1d_dev {

template <typename real>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

constexpr int kStages = 4;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of `bar` with the given parity to complete.  Gives up
// after limit_ns (raising a timeout) or, when `watch` is set, as soon as the
// run has failed elsewhere.
__device__ inline bool mbar_wait(uint64_t* bar, unsigned parity, int* status, int64_t limit_ns, bool watch) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  unsigned spins = 0;
  while (!mbar_test(bar, parity)) {
    if ((++spins & 15u) == 0) {
      if (watch && status_failed(status)) return false;
      if (static_cast<int64_t>(global_timer_ns() - t0) > limit_ns) {
        raise_status(status, HEAT1D_ERR_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_copy_to_shared(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

}  // namespace heat1d_dev

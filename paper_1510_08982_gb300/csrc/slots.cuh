// slots.cuh -- tagged slots: a value travels with its version number.
//
// Each 32-bit half of a value shares a 64-bit word with the version (or
// epoch) it belongs to, so a reader that finds the version it wants in every
// word of a slot holds that version's value, and a slot caught in the middle
// of an update simply does not match yet: no release/acquire pair and no
// separate counter sit between writer and reader.  Used by the per-step
// asynchronous kernel for its edge values.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace heat1d_dev {

// A value as 32-bit words, each carried in a tagged slot word.
template <typename real>
struct Tag;
template <>
struct Tag<double> {
  static constexpr int W = 2;
  __device__ static __forceinline__ void split(double x, uint32_t (&b)[2]) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    b[0] = static_cast<uint32_t>(u);
    b[1] = static_cast<uint32_t>(u >> 32);
  }
  __device__ static __forceinline__ double join(const uint32_t (&b)[2]) {
    return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(b[1]) << 32) | b[0]));
  }
};
template <>
struct Tag<float> {
  static constexpr int W = 1;
  __device__ static __forceinline__ void split(float x, uint32_t (&b)[1]) { b[0] = __float_as_uint(x); }
  __device__ static __forceinline__ float join(const uint32_t (&b)[1]) { return __uint_as_float(b[0]); }
};

// Slot word: version in the high half, 32 value bits in the low half.  The
// empty word (also the byte pattern the host clears the global rings with)
// carries version 0x80808080, below any version a run uses (>= -254).
constexpr unsigned long long kEmptySlot = 0x8080808080808080ull;
__device__ __forceinline__ unsigned long long slot_word(int ver, uint32_t bits) {
  return (static_cast<unsigned long long>(static_cast<uint32_t>(ver)) << 32) | bits;
}
__device__ __forceinline__ int slot_ver(unsigned long long w) { return static_cast<int>(static_cast<uint32_t>(w >> 32)); }

// Slot words in this CTA's shared memory: written by a puller of this CTA or
// by a neighbour CTA of the cluster, so both sides use cluster scope.
__device__ __forceinline__ unsigned long long ld_slot_shared(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.cluster.shared::cta.b64 %0, [%1];"
               : "=l"(v)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p)))
               : "memory");
  return v;
}
__device__ __forceinline__ void st_slot_shared(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.cluster.shared::cta.b64 [%0], %1;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))),
               "l"(v)
               : "memory");
}
// A slot word in a neighbour CTA's shared memory (an address from mapa).
__device__ __forceinline__ void st_slot_cluster(uint32_t addr, unsigned long long v) {
  asm volatile("st.relaxed.cluster.shared::cluster.b64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
// Slot words in global memory (read and written at L2).
__device__ __forceinline__ unsigned long long ld_slot_global(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_slot_global(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

}  // namespace heat1d_dev

// cluster.cuh -- thread-block clusters: distributed shared memory addresses,
// stores into a neighbour CTA's shared memory, cluster-scope flags and the
// cluster barrier, and the launch configuration of a 1-D grid in clusters of
// C consecutive CTAs (CTA s has rank s mod C in its cluster).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace heat1d_dev {

// Address, in the cluster's shared window, of `local` (a shared-memory
// object of this kernel) in the CTA of rank `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* local, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(local))), "r"(rank));
  return r;
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster (the non-aligned form: threads
// may arrive from different code paths; none may have exited before it).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// A value stored into another CTA's shared memory (weak: published by a
// later release).
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// A flag in another CTA's shared memory, released at cluster scope; and its
// acquiring read in the CTA that owns it.
__device__ __forceinline__ void st_release_cluster(uint32_t addr, int v) {
  asm volatile("st.release.cluster.shared::cluster.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cluster_shared(const int* p) {
  int v;
  asm volatile("ld.acquire.cluster.shared::cta.b32 %0, [%1];"
               : "=r"(v)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p)))
               : "memory");
  return v;
}

}  // namespace heat1d_dev

namespace heat1d_impl {

// Launch configuration of a 1-D grid of S CTAs in clusters of C (C > 1).
inline cudaLaunchConfig_t cluster_launch_config(int S, int threads, size_t smem, int C, cudaStream_t st,
                                                cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// The largest of 8, 4, 2 that divides S and lets every cluster of `kernel`
// be resident (else 1), or, for wanted > 1, that size if it qualifies (else
// 0).  wanted == 1 and S < 2 give 1.
template <typename Kernel>
int pick_cluster_size(Kernel kernel, int S, int threads, size_t smem, int wanted) {
  if (wanted == 1 || S < 2) return wanted <= 1 ? 1 : 0;
  const int cands[3] = {8, 4, 2};
  for (int c : cands) {
    if ((wanted && c != wanted) || S % c != 0) continue;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_launch_config(S, threads, smem, c, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (static_cast<int64_t>(n) * c >= S) return c;
  }
  return wanted ? 0 : 1;
}

}  // namespace heat1d_impl

// stream_kernels.cu -- the synchronous run for rods too long to stay on chip:
// temporal blocking with overlapped halos, T steps per pass over HBM.
//
// The rod is cut into tiles of W points.  A pass reads tile j and Th >= T halo
// points on each side from one state buffer, advances the tile T steps in
// registers (the valid region shrinks by one point per side per step -- the
// overlapped-halo trapezoid), and writes its W points to the other buffer.
// Consecutive passes alternate the two buffers.  Halo points are recomputed
// with the same arithmetic, so the result is identical, bit for bit, to K
// single steps of Section 2's Eq. (eqn:sync).
//
// One persistent cooperative launch runs every pass.  CTA c processes tiles
// c, c+G, c+2G, ... in each pass.  Instead of a grid barrier between passes,
// each tile carries a pass counter: tile j may start pass p+1 once tiles j-1
// and j+1 have finished pass p (they then no longer read the buffer tile j is
// about to overwrite, and what tile j reads is complete).  Waits only point to
// earlier passes, so the launch cannot deadlock while all CTAs are resident.
//
// Loads and stores move 16 bytes per thread per instruction where a thread's
// run of E points lies inside the rod (tile starts are 16-byte aligned).
#include <algorithm>

#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

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

// Waits until the pass counter of a neighbouring tile reaches `want`.
__device__ bool wait_tile(const int* done, int want, int* status, int64_t limit_ns) {
  if (ld_acquire_gpu(done) >= want) return true;
  const uint64_t t0 = global_timer_ns();
  unsigned spins = 0;
  while (ld_acquire_gpu(done) < want) {
    if ((++spins & 31u) == 0) {
      if (status_failed(status)) return false;
      if (static_cast<int64_t>(global_timer_ns() - t0) > limit_ns) {
        raise_status(status, HEAT1D_ERR_TIMEOUT);
        return false;
      }
    }
    __nanosleep(64);
  }
  return true;
}

template <typename real, int E>
__global__ void __launch_bounds__(max_tile_threads(sizeof(real), E), 1) stream_kernel(StreamRun a) {
  using V = typename Vec16<real>::type;
  using Win = Window<E, sync_window_halo(sizeof(real), E)>;
  constexpr int VN = Vec16<real>::n;
  static_assert(E % VN == 0, "E must be a multiple of the 16-byte vector width");
  __shared__ WindowShared<real, Win::H> sh;
  __shared__ int sh_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

  const int64_t N = a.N;
  const int Th = a.Th, W = a.W;
  const real c1 = static_cast<real>(a.c1), cN = static_cast<real>(a.cN);
  const Coef<real> coef{static_cast<real>(a.r), static_cast<real>(a.N > 0)};
  real* buf[2] = {static_cast<real*>(a.u_a), static_cast<real*>(a.u_b)};
  const int npass = static_cast<int>((a.K + a.T - 1) / a.T);
  const int p0 = Win::pos(warp, lane, 0);  // this thread's first position
  // lanes 1..30 own all their positions; lanes 0 and 31 may hold halo copies
  const bool owns_all = Win::owner(warp, lane, 0, nwarps) && Win::owner(warp, lane, E - 1, nwarps);
  int parity = 0;

  for (int p = 0; p < npass; ++p) {
    const real* __restrict__ src = buf[p & 1];
    real* __restrict__ dst = buf[(p + 1) & 1];
    const int tb = static_cast<int>(std::min<int64_t>(a.T, a.K - static_cast<int64_t>(p) * a.T));
    for (int64_t j = blockIdx.x; j < a.ntiles; j += gridDim.x) {
      if (p > 0) {
        if (tid == 0) {
          bool ok = true;
          if (j > 0) ok = wait_tile(a.done + (j - 1), p, a.status, a.spin_limit_ns);
          if (ok && j + 1 < a.ntiles) ok = wait_tile(a.done + (j + 1), p, a.status, a.spin_limit_ns);
          sh_ok = ok;
        }
        __syncthreads();
        if (!sh_ok) return;
      }
      // Load: position q holds global point g0 + q, g0 = j*W - Th.
      const int64_t gt = j * W - Th + p0;
      real v[E];
      if (gt >= 0 && gt + E <= N) {
#pragma unroll
        for (int i = 0; i < E / VN; ++i) {
          const V x = __ldcg(reinterpret_cast<const V*>(src + gt) + i);
          const real* xs = reinterpret_cast<const real*>(&x);
#pragma unroll
          for (int q = 0; q < VN; ++q) v[i * VN + q] = xs[q];
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int64_t g = gt + e;
          v[e] = (g >= 0 && g < N) ? __ldcg(src + g) : static_cast<real>(0);
        }
      }
      unsigned fixed = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t g = gt + e;
        if (g == 0) v[e] = c1;
        if (g == N - 1) v[e] = cN;
        if (g <= 0 || g >= N - 1) fixed |= 1u << e;
      }
      const int mode = tile_mode<E>(fixed);
      warp_advance<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwarps, blockDim.x, tb);

      // Store the W own points (positions Th .. Th+W-1) inside the rod.
      if (owns_all && p0 >= Th && p0 + E <= Th + W && gt >= 0 && gt + E <= N) {
#pragma unroll
        for (int i = 0; i < E / VN; ++i) {
          V x;
          real* xs = reinterpret_cast<real*>(&x);
#pragma unroll
          for (int q = 0; q < VN; ++q) xs[q] = v[i * VN + q];
          __stcg(reinterpret_cast<V*>(dst + gt) + i, x);
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int q = p0 + e;
          const int64_t g = gt + e;
          if (q >= Th && q < Th + W && g >= 0 && g < N && Win::owner(warp, lane, e, nwarps)) __stcg(dst + g, v[e]);
        }
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_gpu(a.done + j, p + 1);
      }
    }
  }
}

template <typename real, int E>
int launch_stream_t(const StreamRun& a, int threads, int grid, cudaStream_t st) {
  StreamRun args = a;
  void* params[] = {&args};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(stream_kernel<real, E>), dim3(grid),
                                              dim3(threads), params, 0, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

template <typename real, int E>
int resident_stream_t(int threads) {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_kernel<real, E>, threads, 0) != cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace

int launch_stream(const StreamRun& a, int dtype, int E, int threads, int grid, cudaStream_t st) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 4: return f64 ? launch_stream_t<double, 4>(a, threads, grid, st) : launch_stream_t<float, 4>(a, threads, grid, st);
    case 8: return f64 ? launch_stream_t<double, 8>(a, threads, grid, st) : launch_stream_t<float, 8>(a, threads, grid, st);
    case 16: return f64 ? launch_stream_t<double, 16>(a, threads, grid, st) : launch_stream_t<float, 16>(a, threads, grid, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

int max_resident_stream(int dtype, int E, int threads) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 4: return f64 ? resident_stream_t<double, 4>(threads) : resident_stream_t<float, 4>(threads);
    case 8: return f64 ? resident_stream_t<double, 8>(threads) : resident_stream_t<float, 8>(threads);
    case 16: return f64 ? resident_stream_t<double, 16>(threads) : resident_stream_t<float, 16>(threads);
    default: return 0;
  }
}

}  // namespace heat1d_impl

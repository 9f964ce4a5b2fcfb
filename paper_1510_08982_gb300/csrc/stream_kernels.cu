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
// A tile and its halos arrive in shared memory by one bulk copy (tile starts
// are 16-byte aligned); stores move 16 bytes per thread per instruction where
// a thread's run of E points lies inside the rod.
#include <algorithm>

#include "bulk.cuh"
#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

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

// ------------------------------------------------------------ the pipeline
//
// Tile loads and pass-counter releases are taken off the compute warps' path
// by two extra warps (the stage ring and its mbarriers are in bulk.cuh):
//  - the loader (one thread) waits for a tile's previous pass and its
//    neighbours', then copies the tile and its halos from HBM into one of
//    kStages shared-memory stages with a single bulk copy (cp.async.bulk, the
//    1D form of TMA) whose completion lands on the stage's "full" mbarrier;
//  - the compute warps read the stage into registers, advance the tile, store
//    it and arrive on the stage's "stored" mbarrier;
//  - the releaser (one thread) waits on "stored", makes the tile's stores
//    visible GPU-wide, release-stores the tile's pass counter and hands the
//    stage back to the loader ("free").
// Tiles whose halos reach past either end of the rod are loaded by the
// compute warps with plain loads (the stage is then only a signal).  Every
// wait is bounded; on a failure the loader waits for its own copies before it
// returns.

template <typename real, int E>
__global__ void __launch_bounds__(kStreamMaxThreads + 64, 1) stream_tma_kernel(StreamRun a) {
  using V = typename Vec16<real>::type;
  using Win = Window<E, stream_window_halo(sizeof(real), E)>;
  constexpr int VN = Vec16<real>::n;
  static_assert(E % VN == 0, "E must be a multiple of the 16-byte vector width");
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ WindowShared<real, Win::H> sh;
  __shared__ __align__(8) uint64_t full[kStages], stored[kStages], freed[kStages];
  __shared__ int stage_plain[kStages];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwc = (blockDim.x >> 5) - 2;  // compute warps; then the loader and the releaser warp
  const unsigned nthreads_c = static_cast<unsigned>(nwc) * 32u;
  const int64_t N = a.N;
  const int Th = a.Th, W = a.W, Wt = a.W + 2 * a.Th;
  real* stage0 = reinterpret_cast<real*>(dyn);
  real* buf[2] = {static_cast<real*>(a.u_a), static_cast<real*>(a.u_b)};
  const int npass = static_cast<int>((a.K + a.T - 1) / a.T);
  const int64_t my_tiles = a.ntiles > blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // Items in order: every pass, this CTA's tiles blockIdx.x, blockIdx.x + G, ...
  const int64_t items = my_tiles * npass;

  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&stored[st], static_cast<unsigned>(nwc));
      mbar_init(&freed[st], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == nwc) {  // ------------------------------------------------ loader
    if (lane != 0) return;
    int64_t issued = 0;
    bool ok = true;
    int p = 0, st = 0;
    unsigned round = 0;
    int64_t j = blockIdx.x;
    for (int64_t i = 0; i < items && ok; ++i) {
      if (round > 0 && !mbar_wait(&freed[st], (round - 1) & 1u, a.status, a.spin_limit_ns, true)) break;
      if (p > 0) {
        // The tile's previous pass and its neighbours'.  The tile's own pass
        // was stored by this CTA's compute warps, which the copies run ahead
        // of; when the CTA has at least kStages tiles, the wait on "freed"
        // above already covers it (the releaser works in item order).
        // Acquire loads, not relaxed loads and a GPU-scope fence: measured
        // faster, as such a fence also waits for this thread's copies in
        // flight.
        if (my_tiles < kStages) ok = wait_tile(a.done + j, p, a.status, a.spin_limit_ns);
        if (ok && j > 0) ok = wait_tile(a.done + (j - 1), p, a.status, a.spin_limit_ns);
        if (ok && j + 1 < a.ntiles) ok = wait_tile(a.done + (j + 1), p, a.status, a.spin_limit_ns);
        if (!ok) break;
      }
      const int64_t g0 = j * W - Th;
      const bool plain = g0 < 0 || g0 + Wt > N;
      stage_plain[st] = plain;
      if (plain) {
        mbar_arrive(&full[st]);  // release: the waits above happen before the compute warps' loads
      } else {
        // The neighbours' stores were made through the generic proxy; the copy
        // reads through the async proxy, and the stage's previous contents
        // were read through the generic proxy.
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const unsigned bytes = static_cast<unsigned>(Wt) * sizeof(real);
        mbar_arrive_expect_tx(&full[st], bytes);
        bulk_copy_to_shared(stage0 + static_cast<size_t>(st) * Wt, buf[p & 1] + g0, bytes, &full[st]);
      }
      issued = i + 1;
      j += gridDim.x;
      if (j >= a.ntiles) {
        j = blockIdx.x;
        ++p;
      }
      if (++st == kStages) {
        st = 0;
        ++round;
      }
    }
    // Copies still in flight (only after a failure) must land before the CTA leaves.
    for (int64_t i = issued > kStages ? issued - kStages : 0; i < issued; ++i)
      mbar_wait(&full[i % kStages], static_cast<unsigned>(i / kStages) & 1u, a.status, a.spin_limit_ns, false);
    return;
  }

  if (warp == nwc + 1) {  // -------------------------------------------- releaser
    if (lane != 0) return;
    int p = 0, st = 0;
    unsigned round = 0;
    int64_t j = blockIdx.x;
    for (int64_t i = 0; i < items; ++i) {
      if (!mbar_wait(&stored[st], round & 1u, a.status, a.spin_limit_ns, true)) break;
      // The compute warps' stores, ordered before their arrivals (release at
      // CTA scope, acquired by the wait above), are ordered before the
      // counter by this release at GPU scope (cumulativity).  No separate
      // fence: it would wait a second time for the same stores.
      if (j != a.stall_tile) st_release_gpu(a.done + j, p + 1);
      mbar_arrive(&freed[st]);
      j += gridDim.x;
      if (j >= a.ntiles) {
        j = blockIdx.x;
        ++p;
      }
      if (++st == kStages) {
        st = 0;
        ++round;
      }
    }
    return;
  }

  // ------------------------------------------------------------ compute warps
  const Coef<real> coef{kparam<real>(a.r, a.r_f), kparam<real>(a.one, a.one_f)};
  const real c1 = kparam<real>(a.c1, a.c1_f), cN = kparam<real>(a.cN, a.cN_f);
  const int p0 = Win::pos(warp, lane, 0);
  const bool owns_all = Win::owner(warp, lane, 0, nwc) && Win::owner(warp, lane, E - 1, nwc);
  int parity = 0;
  int p = 0, st = 0;
  unsigned round = 0;
  int64_t j = blockIdx.x;
  for (int64_t i = 0; i < items; ++i) {
    const real* __restrict__ src = buf[p & 1];
    real* __restrict__ dst = buf[(p + 1) & 1];
    const int tb = static_cast<int>(std::min<int64_t>(a.T, a.K - static_cast<int64_t>(p) * a.T));
    bool failed = !mbar_wait(&full[st], round & 1u, a.status, a.spin_limit_ns, true);
    const int64_t g0 = j * W - Th;
    const int64_t gt = g0 + p0;
    // A tile clear of both ends of the rod (the common case) has no fixed
    // point, every window position inside the rod and an in-range store.
    const bool inner = g0 > 0 && g0 + Wt < N;
    real v[E];
    if (!failed && !stage_plain[st]) {
      const real* sp = stage0 + static_cast<size_t>(st) * Wt + p0;
#pragma unroll
      for (int q = 0; q < E / VN; ++q) {
        const V x = reinterpret_cast<const V*>(sp)[q];
        const real* xs = reinterpret_cast<const real*>(&x);
#pragma unroll
        for (int t = 0; t < VN; ++t) v[q * VN + t] = xs[t];
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t g = gt + e;
        v[e] = (!failed && g >= 0 && g < N) ? __ldcg(src + g) : static_cast<real>(0);
      }
    }
    // A failed wait ends the run for every compute warp.  Passes longer than
    // H steps meet halo-refresh barriers, so there the warps leave together;
    // shorter passes meet none (the last refresh of a pass is left out) and
    // each warp may leave on its own.
    if (a.T > Win::H) {
      if (named_barrier_or(2, nthreads_c, failed)) return;
    } else if (failed) {
      return;
    }
    if (inner) {
      warp_advance<real, E, Win::H>(kTileFree, v, 0u, coef, sh, parity, warp, lane, nwc, nthreads_c, tb, false);
    } else {
      unsigned fixed = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int64_t g = gt + e;
        if (g == 0) v[e] = c1;
        if (g == N - 1) v[e] = cN;
        if (g <= 0 || g >= N - 1) fixed |= 1u << e;
      }
      const int mode = tile_mode<E>(fixed);
      warp_advance<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwc, nthreads_c, tb, false);
    }
    if (owns_all && p0 >= Th && p0 + E <= Th + W && (inner || (gt >= 0 && gt + E <= N))) {
#pragma unroll
      for (int q = 0; q < E / VN; ++q) {
        V x;
        real* xs = reinterpret_cast<real*>(&x);
#pragma unroll
        for (int t = 0; t < VN; ++t) xs[t] = v[q * VN + t];
        __stcg(reinterpret_cast<V*>(dst + gt) + q, x);
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int qq = p0 + e;
        const int64_t g = gt + e;
        if (qq >= Th && qq < Th + W && g >= 0 && g < N && Win::owner(warp, lane, e, nwc)) __stcg(dst + g, v[e]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&stored[st]);  // release: this warp's stores come first
    j += gridDim.x;
    if (j >= a.ntiles) {
      j = blockIdx.x;
      ++p;
    }
    if (++st == kStages) {
      st = 0;
      ++round;
    }
  }
}

template <typename real, int E>
size_t tma_smem_bytes(int Wt) {
  return static_cast<size_t>(kStages) * Wt * sizeof(real);
}

template <typename real, int E>
int launch_stream_tma_t(const StreamRun& a, int threads, int grid, cudaStream_t st) {
  StreamRun args = a;
  set_run_params(args);
  void* params[] = {&args};
  const size_t smem = tma_smem_bytes<real, E>(a.W + 2 * a.Th);
  if (cudaFuncSetAttribute(stream_tma_kernel<real, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return HEAT1D_ERR_CUDA;
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(stream_tma_kernel<real, E>), dim3(grid),
                                              dim3(threads + 64), params, smem, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

template <typename real, int E>
int resident_stream_tma_t(int threads, int Wt) {
  int per_sm = 0, dev = 0, nsm = 0;
  const size_t smem = tma_smem_bytes<real, E>(Wt);
  if (cudaFuncSetAttribute(stream_tma_kernel<real, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_tma_kernel<real, E>, threads + 64, smem) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace

int launch_stream_tma(const StreamRun& a, int dtype, int E, int threads, int grid, cudaStream_t st) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 4: return f64 ? launch_stream_tma_t<double, 4>(a, threads, grid, st) : launch_stream_tma_t<float, 4>(a, threads, grid, st);
    case 8: return f64 ? launch_stream_tma_t<double, 8>(a, threads, grid, st) : launch_stream_tma_t<float, 8>(a, threads, grid, st);
    case 16: return f64 ? launch_stream_tma_t<double, 16>(a, threads, grid, st) : launch_stream_tma_t<float, 16>(a, threads, grid, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

int max_resident_stream_tma(int dtype, int E, int threads, int Wt) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 4: return f64 ? resident_stream_tma_t<double, 4>(threads, Wt) : resident_stream_tma_t<float, 4>(threads, Wt);
    case 8: return f64 ? resident_stream_tma_t<double, 8>(threads, Wt) : resident_stream_tma_t<float, 8>(threads, Wt);
    case 16: return f64 ? resident_stream_tma_t<double, 16>(threads, Wt) : resident_stream_tma_t<float, 16>(threads, Wt);
    default: return 0;
  }
}

}  // namespace heat1d_impl

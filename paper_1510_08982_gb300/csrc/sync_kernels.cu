// sync_kernels.cu -- the synchronous run of Section 2, Eq. (eqn:sync), as one
// persistent cooperative launch.
//
// The paper's synchronous code relaunches a kernel (and copies the state to
// the host and back) every step; Section 4 names __syncthreads() as the better
// way to impose the per-step synchronisation.  Here one CTA owns one segment
// (the PE of Fig. 1) for the whole run.  The segment and T halo points on each
// side live in registers.  The CTA advances T steps on its own (the valid region
// shrinks by one point per side per step, the overlapped-halo trapezoid), then
// publishes its first and last T points, meets every other CTA at a grid-wide
// barrier, and reloads its halos from its neighbours.  Halo points are
// recomputed redundantly with the same arithmetic, so the result is identical,
// bit for bit, to a barrier after every step (T = 1).
#include <algorithm>

#include "checked.cuh"
#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

// Grid barrier on a counter that starts at zero: arrival number `epoch`
// (0-based) completes when the counter reaches S*(epoch+1).  Called by one
// thread per CTA between two __syncthreads().  The arrival is a release
// reduction (it orders the CTA's edge stores, seen through the CTA barrier,
// before it) and the wait an acquire load that reads the last arrival (every
// arrival is a release on the same counter), so no separate fences.  Returns
// false on a timeout or a failure raised elsewhere.
__device__ bool grid_barrier(unsigned* counter, unsigned target, int* status, int64_t limit_ns) {
  red_release_gpu_add(counter, 1u);
  const uint64_t t0 = global_timer_ns();
  unsigned spins = 0;
  while (true) {
    const unsigned c = ld_acquire_gpu_u32(counter);
    if (static_cast<int>(c - target) >= 0) break;
    if ((++spins & 63u) == 0) {
      if (status_failed(status)) return false;
      if (static_cast<int64_t>(global_timer_ns() - t0) > limit_ns) {
        raise_status(status, HEAT1D_ERR_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

template <typename real, int E>
__global__ void __launch_bounds__(max_tile_threads(sizeof(real), E), 1) sync_persistent_kernel(SegmentRun a) {
  using Win = Window<E, sync_window_halo(sizeof(real), E)>;
  __shared__ WindowShared<real, Win::H> sh;
  __shared__ int sh_ok;
  const int s = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t N = a.N;
  const int64_t a0 = a.seg_off[s];
  const int L = static_cast<int>(a.seg_off[s + 1] - a0);
  const int T = a.T;
  const real c1 = kparam<real>(a.c1, a.c1_f), cN = kparam<real>(a.cN, a.cN_f);
  const Coef<real> coef{kparam<real>(a.r, a.r_f), kparam<real>(a.one, a.one_f)};  // one = 1 at run time
  const real* __restrict__ uin = static_cast<const real*>(a.u_in);
  real* __restrict__ uout = static_cast<real*>(a.u_out);
  real* edges = static_cast<real*>(a.edges);
  const bool first = !a.periodic && s == 0;        // holds the Dirichlet end u_1
  const bool last = !a.periodic && s == a.S - 1;   // holds the Dirichlet end u_N

  // Tile layout: position p holds global point a0 - lo + p; the owned points
  // are [lo, hi), the left halo [lo - T, lo), the right halo [hi, hi + T).
  // Interior segments: lo = T.  The first segment has no left halo (lo = 0),
  // so that u_1 sits in slot 0 of lane 0 of warp 0; the last segment ends at
  // the last position the CTA covers, so that u_N sits in slot E-1 of lane 31
  // of the last warp (its positions left of the halo are stepped but never
  // read by an owned point within a block).  Both ends are then held by two
  // selects per step in those two warps instead of a select per point.  With
  // a single segment u_N falls wherever the rod ends.
  const int P = nwarps * Win::D + 2 * Win::H;  // positions the CTA covers
  const int lo = first ? 0 : (last ? P - L : T);
  const int hi = lo + L;
  const int tile_end = last ? hi : hi + T;     // positions past it are padding
  real v[E];
  unsigned fixed = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = Win::pos(warp, lane, e);
    const int64_t g = a0 - lo + p;
    real x = static_cast<real>(0);
    if (a.periodic) {  // halos wrap around the ring
      const int64_t gw = ((g % N) + N) % N;
      if (p < tile_end && index_ok(a.status, gw, N)) x = uin[gw];
    } else {
      if (p < tile_end && g >= 0 && g < N && index_ok(a.status, g, N)) x = uin[g];
      if (g == 0) x = c1;
      if (g == N - 1) x = cN;
      if (p < tile_end && (g == 0 || g == N - 1)) fixed |= 1u << e;
    }
    v[e] = x;
  }
  const int sl = s > 0 ? s - 1 : (a.periodic ? a.S - 1 : -1);      // left neighbour segment
  const int sr = s + 1 < a.S ? s + 1 : (a.periodic ? 0 : -1);       // right neighbour segment
  const int mode = Win::pos(warp, 0, 0) >= tile_end ? static_cast<int>(kTileIdle) : tile_mode<E>(fixed);

  if (a.snap) {  // row 0: the state at step 0
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = Win::pos(warp, lane, e);
      if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps) && index_ok(a.status, a0 + (p - lo), a.snap_len))
        static_cast<real*>(a.snap)[a0 + (p - lo)] = v[e];
    }
  }
  int parity = 0;
  unsigned epoch = 0;
  for (int64_t k0 = 0; k0 < a.K; k0 += T) {
    const int tb = static_cast<int>(std::min<int64_t>(T, a.K - k0));
    warp_advance<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwarps, blockDim.x, tb);
    if (a.snap && (k0 + tb) % a.snap_every == 0) {  // owners record the state at step k0+tb
      const int64_t row0 = ((k0 + tb) / a.snap_every) * N;
      real* row = static_cast<real*>(a.snap) + row0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps) && index_ok(a.status, row0 + a0 + (p - lo), a.snap_len))
          row[a0 + (p - lo)] = v[e];
      }
    }
    if (k0 + tb >= a.K) break;

    // Publish the first T and the last T points of the segment.
    const int64_t mine0 = (static_cast<int64_t>(epoch & 1u) * a.S + s) * 2 * T;
    real* mine = edges + mine0;
    if (Win::touches(warp, lo, lo + T) || Win::touches(warp, hi - T, hi)) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (!Win::owner(warp, lane, e, nwarps)) continue;
        if (p >= lo && p < lo + T && index_ok(a.status, mine0 + (p - lo), a.edges_len)) st_cg(mine + (p - lo), v[e]);
        if (p >= hi - T && p < hi && index_ok(a.status, mine0 + T + (p - (hi - T)), a.edges_len))
          st_cg(mine + T + (p - (hi - T)), v[e]);
      }
    }
    __syncthreads();
    if (tid == 0) {
      sh_ok = grid_barrier(a.barrier, static_cast<unsigned>(a.S) * (epoch + 1u), a.status, a.spin_limit_ns);
    }
    __syncthreads();
    if (!sh_ok) return;  // CTA-uniform: every thread reads the same flag

    // Reload the halos (every copy): the left neighbour's last T points, the
    // right neighbour's first T points.
    if (sl >= 0 && Win::touches(warp, lo - T, lo)) {
      const int64_t left0 = (static_cast<int64_t>(epoch & 1u) * a.S + sl) * 2 * T + T;
      const real* left = edges + left0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (p >= lo - T && p < lo && index_ok(a.status, left0 + (p - (lo - T)), a.edges_len))
          v[e] = ld_cg(left + (p - (lo - T)));
      }
    }
    if (sr >= 0 && Win::touches(warp, hi, hi + T)) {
      const int64_t right0 = (static_cast<int64_t>(epoch & 1u) * a.S + sr) * 2 * T;
      const real* right = edges + right0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (p >= hi && p < hi + T && index_ok(a.status, right0 + (p - hi), a.edges_len)) v[e] = ld_cg(right + (p - hi));
      }
    }
    ++epoch;
  }

#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = Win::pos(warp, lane, e);
    if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps) && index_ok(a.status, a0 + (p - lo), N))
      uout[a0 + (p - lo)] = v[e];
  }
}

template <typename real, int E>
int launch_sync_t(const SegmentRun& a, int threads, cudaStream_t st) {
  SegmentRun args = a;
  set_run_params(args);
  void* params[] = {&args};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(sync_persistent_kernel<real, E>), dim3(a.S),
                                              dim3(threads), params, 0, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

template <typename real, int E>
int resident_t(int threads) {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sync_persistent_kernel<real, E>, threads, 0) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace

int launch_sync_persistent(const SegmentRun& a, int dtype, int E, int threads, cudaStream_t st) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 2: return f64 ? launch_sync_t<double, 2>(a, threads, st) : launch_sync_t<float, 2>(a, threads, st);
    case 4: return f64 ? launch_sync_t<double, 4>(a, threads, st) : launch_sync_t<float, 4>(a, threads, st);
    case 8: return f64 ? launch_sync_t<double, 8>(a, threads, st) : launch_sync_t<float, 8>(a, threads, st);
    case 16: return f64 ? launch_sync_t<double, 16>(a, threads, st) : launch_sync_t<float, 16>(a, threads, st);
    case 32: return f64 ? HEAT1D_ERR_INVAL : launch_sync_t<float, 32>(a, threads, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

int max_resident_sync(int dtype, int E, int threads) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 2: return f64 ? resident_t<double, 2>(threads) : resident_t<float, 2>(threads);
    case 4: return f64 ? resident_t<double, 4>(threads) : resident_t<float, 4>(threads);
    case 8: return f64 ? resident_t<double, 8>(threads) : resident_t<float, 8>(threads);
    case 16: return f64 ? resident_t<double, 16>(threads) : resident_t<float, 16>(threads);
    case 32: return f64 ? 0 : resident_t<float, 32>(threads);
    default: return 0;
  }
}

}  // namespace heat1d_impl

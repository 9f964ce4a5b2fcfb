// blocked_kernels.cu -- the asynchronous run with temporal blocking: the
// bounded-delay model of Section 3 with blocks of T steps in place of single
// steps.
//
// One CTA owns one segment (the PE of Fig. 1) for the whole run and holds it,
// with T halo points per side, in registers, exactly as the synchronous
// persistent kernel does.  Block b advances T steps on that tile (the valid
// region shrinks by one point per side per step).  Where the synchronous
// kernel then meets every CTA at a grid barrier, this one publishes its first
// and last T points as strip version b+1 into a ring of R strips, release-stores
// its version counter, and starts block b+1 with the newest strip of each
// neighbour that is not newer than b+1 -- waiting only while that strip is
// more than q-1 blocks old.  The delay d = (b+1) - v of every strip read is
// recorded, and a replay waits for exactly v = b+1 - d.  On the periodic
// ring (Section 5.3) the neighbours of the end segments are each other.
//
// Ring safety: a segment cannot start block b before both neighbours have
// published version b-q+1, so neighbours drift at most q-1 blocks apart; a
// reader in block b' needs versions >= b'-q+1 while a writer in block b <=
// b'+q-1 overwrites version b+1-R, which is older whenever R >= 2q.
#include <algorithm>

#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

// Chooses (free run) or looks up (replay) the neighbour strip version that
// block j reads, waiting for it with a bounded spin.  Called by one thread.
// Returns the version, or -1 after raising a failure.
__device__ int strip_version(const SegmentRun& a, const int* nb_prog, int j, size_t tidx) {
  int need;
  if (a.trace_in) {
    const int d = a.trace_in[tidx];
    if (d >= a.q) {
      raise_status(a.status, HEAT1D_ERR_TRACE);
      return -1;
    }
    need = j - min(d, j);
  } else {
    need = max(j - a.q + 1, 0);
  }
  int V = ld_acquire_gpu(nb_prog);
  if (V < need) {
    const uint64_t t0 = global_timer_ns();
    unsigned spins = 0;
    while ((V = ld_acquire_gpu(nb_prog)) < need) {
      if ((++spins & 63u) == 0) {
        if (status_failed(a.status)) return -1;
        if (static_cast<int64_t>(global_timer_ns() - t0) > a.spin_limit_ns) {
          raise_status(a.status, HEAT1D_ERR_TIMEOUT);
          return -1;
        }
      }
    }
  }
  const int v = a.trace_in ? need : min(V, j);
  if (a.trace_out) a.trace_out[tidx] = static_cast<uint8_t>(j - v);
  return v;
}

// Stores the segment's first and last T points as strip version `ver`, then
// (one thread, after the CTA barrier) release-stores the version counter.
template <typename real, int E, typename Win>
__device__ __forceinline__ void publish_strips(const real (&v)[E], real* strips, int* my_prog, int s, int R, int T,
                                               int lo, int hi, int ver, bool stalled, int warp, int lane, int nwarps,
                                               int tid) {
  real* mine = strips + (static_cast<size_t>(s) * R + (ver & (R - 1))) * 2 * T;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = Win::pos(warp, lane, e);
    if (!Win::owner(warp, lane, e, nwarps)) continue;
    if (p >= lo && p < lo + T) st_cg(mine + (p - lo), v[e]);
    if (p >= hi - T && p < hi) st_cg(mine + T + (p - (hi - T)), v[e]);
  }
  __syncthreads();
  // A release at GPU scope after the CTA barrier orders every thread's strip
  // stores before the version (cumulativity); no separate fence.
  if (tid == 0 && !stalled) st_release_gpu(my_prog, ver);
}

template <typename real, int E>
__global__ void __launch_bounds__(max_tile_threads(sizeof(real), E), 1) async_blocked_kernel(SegmentRun a) {
  using Win = Window<E, sync_window_halo(sizeof(real), E)>;
  __shared__ WindowShared<real, Win::H> sh;
  __shared__ int sh_v[2];  // strip versions read by this block: [0] left, [1] right (-1: failed)
  const int s = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int64_t N = a.N;
  const int64_t a0 = a.seg_off[s];
  const int L = static_cast<int>(a.seg_off[s + 1] - a0);
  const int T = a.T, R = a.R, S = a.S;
  const real c1 = kparam<real>(a.c1, a.c1_f), cN = kparam<real>(a.cN, a.cN_f);
  const Coef<real> coef{kparam<real>(a.r, a.r_f), kparam<real>(a.one, a.one_f)};  // one = 1 at run time
  const real* __restrict__ uin = static_cast<const real*>(a.u_in);
  real* __restrict__ uout = static_cast<real*>(a.u_out);
  real* strips = static_cast<real*>(a.rings);  // [S][R][2T]: first T points, last T points
  int* my_prog = a.prog + static_cast<size_t>(s) * kProgStride;
  const bool stalled = s == a.stall_segment;
  const bool periodic = a.periodic != 0;
  const int sl = s > 0 ? s - 1 : (periodic ? S - 1 : -1);  // neighbours (ring when periodic)
  const int sr = s + 1 < S ? s + 1 : (periodic ? 0 : -1);
  const int nbnd = periodic ? S : S - 1;                    // boundaries: S on the ring
  const int bl = periodic ? (s + S - 1) % S : s - 1;        // boundary read on the left (side 1)

  // Tile layout as in the synchronous kernel: position p holds global point
  // a0 - lo + p, owned points [lo, hi), halos [lo - T, lo) and [hi, hi + T);
  // the first segment starts at u_1 (lo = 0) and the last one ends at u_N in
  // the CTA's last position, so that both Dirichlet ends sit in slots known
  // at compile time (block 0: every strip is version 0, the initial state).
  const bool first = !periodic && s == 0, last = !periodic && s == S - 1;
  const int P = nwarps * Win::D + 2 * Win::H;
  const int lo = first ? 0 : (last ? P - L : T);
  const int hi = lo + L;
  const int tile_end = last ? hi : hi + T;
  real v[E];
  unsigned fixed = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = Win::pos(warp, lane, e);
    const int64_t g = a0 - lo + p;
    real x = static_cast<real>(0);
    if (periodic) {  // halos wrap around the ring
      if (p < tile_end) x = uin[((g % N) + N) % N];
    } else {
      if (p < tile_end && g >= 0 && g < N) x = uin[g];
      if (g == 0) x = c1;
      if (g == N - 1) x = cN;
      if (p < tile_end && (g == 0 || g == N - 1)) fixed |= 1u << e;
    }
    v[e] = x;
  }
  const int mode = Win::pos(warp, 0, 0) >= tile_end ? static_cast<int>(kTileIdle) : tile_mode<E>(fixed);

  if (a.snap) {  // row 0: the state at step 0
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = Win::pos(warp, lane, e);
      if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps)) static_cast<real*>(a.snap)[a0 + (p - lo)] = v[e];
    }
  }
  publish_strips<real, E, Win>(v, strips, my_prog, s, R, T, lo, hi, 0, stalled, warp, lane, nwarps, tid);
  int parity = 0;
  int j = 0;
  for (int64_t k0 = 0; k0 < a.K; k0 += T, ++j) {
    // Strip versions for block j: thread 0 the left neighbour, thread 32 the right one.
    if (tid == 0 || tid == 32) {
      const bool left = tid == 0;
      const int nb = left ? sl : sr;
      int ver = j;
      if (nb >= 0) {
        const size_t tidx = (static_cast<size_t>(j) * nbnd + (left ? bl : s)) * 2 + (left ? 1 : 0);
        ver = strip_version(a, a.prog + static_cast<size_t>(nb) * kProgStride, j, tidx);
      }
      sh_v[left ? 0 : 1] = ver;
    }
    if (blockDim.x <= 32 && tid == 0) {  // one-warp CTA: thread 0 takes both sides
      int ver = j;
      if (sr >= 0) {
        const size_t tidx = (static_cast<size_t>(j) * nbnd + s) * 2 + 0;
        ver = strip_version(a, a.prog + static_cast<size_t>(sr) * kProgStride, j, tidx);
      }
      sh_v[1] = ver;
    }
    __syncthreads();
    const int vl = sh_v[0], vr = sh_v[1];
    if (vl < 0 || vr < 0) return;  // CTA-uniform: every thread reads the same words
    if (j > 0) {  // block 0 runs on the initial halos (version 0)
      if (sl >= 0) {
        const real* left = strips + (static_cast<size_t>(sl) * R + (vl & (R - 1))) * 2 * T;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = Win::pos(warp, lane, e);
          if (p >= lo - T && p < lo) v[e] = ld_cg(left + T + (p - (lo - T)));
        }
      }
      if (sr >= 0) {
        const real* right = strips + (static_cast<size_t>(sr) * R + (vr & (R - 1))) * 2 * T;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = Win::pos(warp, lane, e);
          if (p >= hi && p < hi + T) v[e] = ld_cg(right + (p - hi));
        }
      }
    }
    const int tb = static_cast<int>(std::min<int64_t>(T, a.K - k0));
    warp_advance<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwarps, blockDim.x, tb);
    if (a.snap && (k0 + tb) % a.snap_every == 0) {  // owners record the state at step k0+tb
      real* row = static_cast<real*>(a.snap) + static_cast<size_t>((k0 + tb) / a.snap_every) * N;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps)) row[a0 + (p - lo)] = v[e];
      }
    }
    if (k0 + tb >= a.K) break;
    // The barrier inside also keeps sh_v stable until every thread has read it.
    publish_strips<real, E, Win>(v, strips, my_prog, s, R, T, lo, hi, j + 1, stalled, warp, lane, nwarps, tid);
  }

#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = Win::pos(warp, lane, e);
    if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps)) uout[a0 + (p - lo)] = v[e];
  }
}

template <typename real, int E>
int launch_t(const SegmentRun& a, int threads, cudaStream_t st) {
  SegmentRun args = a;
  set_run_params(args);
  void* params[] = {&args};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(async_blocked_kernel<real, E>), dim3(a.S),
                                              dim3(threads), params, 0, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

}  // namespace

int launch_async_blocked(const SegmentRun& a, int dtype, int E, int threads, cudaStream_t st) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 2: return f64 ? launch_t<double, 2>(a, threads, st) : launch_t<float, 2>(a, threads, st);
    case 4: return f64 ? launch_t<double, 4>(a, threads, st) : launch_t<float, 4>(a, threads, st);
    case 8: return f64 ? launch_t<double, 8>(a, threads, st) : launch_t<float, 8>(a, threads, st);
    case 16: return f64 ? launch_t<double, 16>(a, threads, st) : launch_t<float, 16>(a, threads, st);
    case 32: return f64 ? HEAT1D_ERR_INVAL : launch_t<float, 32>(a, threads, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

}  // namespace heat1d_impl

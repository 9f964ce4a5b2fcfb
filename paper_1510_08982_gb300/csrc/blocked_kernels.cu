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
//
// Thread-block clusters: a neighbour in the same cluster receives the strips
// straight into its own shared memory (distributed shared memory: each owner
// thread stores its point into the neighbour CTA's strip ring, then, after
// the CTA barrier, one thread release-stores the neighbour's strip version at
// cluster scope), and reads them there after one acquire on its own shared
// memory.  Neighbours in different clusters keep the rings in global memory.
#include <algorithm>

#include "checked.cuh"
#include "cluster.cuh"
#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

// Chooses (free run) or looks up (replay) the neighbour strip version that
// block j reads, waiting for it with a bounded spin on the neighbour's
// version counter in global memory, or (local = true) on the version word in
// this CTA's shared memory that a neighbour in the cluster releases.  Called
// by one thread.  Returns the version, or -1 after raising a failure.
__device__ int strip_version(const SegmentRun& a, const int* nb_prog, bool local, int j, size_t tidx) {
  int need;
  if (a.trace_in) {
    const int d = index_ok(a.status, static_cast<int64_t>(tidx), a.trace_len) ? a.trace_in[tidx] : 0;
    if (d >= a.q) {
      raise_status(a.status, HEAT1D_ERR_TRACE);
      return -1;
    }
    need = j - min(d, j);
  } else {
    need = max(j - a.q + 1, 0);
  }
  int V = local ? ld_acquire_cluster_shared(nb_prog) : ld_acquire_gpu(nb_prog);
  if (V < need) {
    const uint64_t t0 = global_timer_ns();
    unsigned spins = 0;
    while ((V = local ? ld_acquire_cluster_shared(nb_prog) : ld_acquire_gpu(nb_prog)) < need) {
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
  if (a.trace_out && index_ok(a.status, static_cast<int64_t>(tidx), a.trace_len))
    a.trace_out[tidx] = static_cast<uint8_t>(j - v);
  return v;
}

// Stores the segment's first and last T points as strip version `ver`, then
// (one thread, after the CTA barrier) release-stores the version counter.
// Where the strips go: the global ring (when a neighbour outside the cluster
// reads them) and, for neighbours inside the cluster, the cluster addresses
// of their strip rings and version words (0: not in the cluster).
struct StripOut {
  bool global;
  uint32_t l_ring, l_ver;  // left neighbour's right-strip ring [R][T] and its version word
  uint32_t r_ring, r_ver;  // right neighbour's left-strip ring and version word
};

template <typename real, int E, typename Win>
__device__ __forceinline__ void publish_strips(const real (&v)[E], real* strips, int* my_prog, const StripOut& o,
                                               int s, int R, int T, int lo, int hi, int ver, bool stalled, int warp,
                                               int lane, int nwarps, int tid, int* status, int64_t strips_len) {
  if (!stalled) {
    const int64_t mine0 = (static_cast<int64_t>(s) * R + (ver & (R - 1))) * 2 * T;
    real* mine = strips + mine0;
    const uint32_t slot = static_cast<uint32_t>((ver & (R - 1)) * T * sizeof(real));
    if (Win::touches(warp, lo, lo + T) || Win::touches(warp, hi - T, hi)) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (!Win::owner(warp, lane, e, nwarps)) continue;
        if (p >= lo && p < lo + T) {
          if (o.global && index_ok(status, mine0 + (p - lo), strips_len)) st_cg(mine + (p - lo), v[e]);
          if (o.l_ring) st_cluster(o.l_ring + slot + static_cast<uint32_t>((p - lo) * sizeof(real)), v[e]);
        }
        if (p >= hi - T && p < hi) {
          if (o.global && index_ok(status, mine0 + T + (p - (hi - T)), strips_len))
            st_cg(mine + T + (p - (hi - T)), v[e]);
          if (o.r_ring) st_cluster(o.r_ring + slot + static_cast<uint32_t>((p - (hi - T)) * sizeof(real)), v[e]);
        }
      }
    }
  }
  __syncthreads();
  // A release after the CTA barrier orders every thread's strip stores before
  // the version (cumulativity); no separate fence.
  if (tid == 0 && !stalled) {
    if (o.global) st_release_gpu(my_prog, ver);
    if (o.l_ver) st_release_cluster(o.l_ver, ver);
    if (o.r_ver) st_release_cluster(o.r_ver, ver);
  }
}

template <typename real, int E>
__global__ void __launch_bounds__(max_tile_threads(sizeof(real), E), 1) async_blocked_kernel(SegmentRun a) {
  using Win = Window<E, sync_window_halo(sizeof(real), E)>;
  __shared__ WindowShared<real, Win::H> sh;
  __shared__ int sh_v[2];   // strip versions read by this block: [0] left, [1] right (-1: failed)
  __shared__ int sh_nv[2];  // newest strip version held in lstrip [0] / rstrip [1] (written by cluster neighbours)
  // Strip rings of the neighbours in the cluster, [R][T] each (dynamic shared
  // memory, present only in cluster launches): lstrip the left neighbour's
  // last T points, rstrip the right neighbour's first T points.
  extern __shared__ __align__(16) unsigned char blocked_dyn[];
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
  // Neighbours in this CTA's cluster (a 1-D grid in clusters of C consecutive
  // CTAs; on the periodic ring the two ends only when one cluster holds every
  // segment).
  const int C = a.cluster;
  const unsigned rank = C > 1 ? cluster_rank() : 0u;
  const bool l_intra = C > 1 && sl >= 0 && (rank > 0 || C == S);
  const bool r_intra = C > 1 && sr >= 0 && (static_cast<int>(rank) + 1 < C || C == S);
  real* lstrip = reinterpret_cast<real*>(blocked_dyn);
  real* rstrip = lstrip + static_cast<size_t>(R) * T;
  if (tid == 0) {
    sh_nv[0] = -1;
    sh_nv[1] = -1;
  }
  __syncthreads();
  // No CTA of the cluster may publish into a neighbour before that neighbour
  // has reset its version words.
  if (C > 1) cluster_sync_all();
  StripOut out{(sl >= 0 && !l_intra) || (sr >= 0 && !r_intra), 0u, 0u, 0u, 0u};
  if (l_intra) {
    const unsigned rl = rank == 0 ? static_cast<unsigned>(C - 1) : rank - 1;
    out.l_ring = cluster_addr(rstrip, rl);
    out.l_ver = cluster_addr(&sh_nv[1], rl);
  }
  if (r_intra) {
    const unsigned rr = static_cast<int>(rank) + 1 == C ? 0u : rank + 1;
    out.r_ring = cluster_addr(lstrip, rr);
    out.r_ver = cluster_addr(&sh_nv[0], rr);
  }

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
  const int mode = Win::pos(warp, 0, 0) >= tile_end ? static_cast<int>(kTileIdle) : tile_mode<E>(fixed);

  if (a.snap) {  // row 0: the state at step 0
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = Win::pos(warp, lane, e);
      if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps) && index_ok(a.status, a0 + (p - lo), a.snap_len))
        static_cast<real*>(a.snap)[a0 + (p - lo)] = v[e];
    }
  }
  publish_strips<real, E, Win>(v, strips, my_prog, out, s, R, T, lo, hi, 0, stalled, warp, lane, nwarps, tid, a.status,
                               a.ring_len);
  int parity = 0;
  bool ok = true;
  int j = 0;
  for (int64_t k0 = 0; k0 < a.K; k0 += T, ++j) {
    // Strip versions for block j: thread 0 the left neighbour, thread 32 the right one.
    if (tid == 0 || tid == 32) {
      const bool left = tid == 0;
      const int nb = left ? sl : sr;
      int ver = j;
      if (nb >= 0) {
        const size_t tidx = (static_cast<size_t>(j) * nbnd + (left ? bl : s)) * 2 + (left ? 1 : 0);
        const bool intra = left ? l_intra : r_intra;
        ver = strip_version(a, intra ? &sh_nv[left ? 0 : 1] : a.prog + static_cast<size_t>(nb) * kProgStride, intra,
                            j, tidx);
      }
      sh_v[left ? 0 : 1] = ver;
    }
    if (blockDim.x <= 32 && tid == 0) {  // one-warp CTA: thread 0 takes both sides
      int ver = j;
      if (sr >= 0) {
        const size_t tidx = (static_cast<size_t>(j) * nbnd + s) * 2 + 0;
        ver = strip_version(a, r_intra ? &sh_nv[1] : a.prog + static_cast<size_t>(sr) * kProgStride, r_intra, j,
                            tidx);
      }
      sh_v[1] = ver;
    }
    __syncthreads();
    const int vl = sh_v[0], vr = sh_v[1];
    if (vl < 0 || vr < 0) {  // CTA-uniform: every thread reads the same words
      ok = false;
      break;
    }
    if (j > 0) {  // block 0 runs on the initial halos (version 0)
      if (sl >= 0 && Win::touches(warp, lo - T, lo)) {
        const int64_t left0 = (static_cast<int64_t>(sl) * R + (vl & (R - 1))) * 2 * T + T;
        const real* left = strips + left0;
        const real* lloc = lstrip + static_cast<size_t>(vl & (R - 1)) * T;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = Win::pos(warp, lane, e);
          if (p >= lo - T && p < lo && (l_intra || index_ok(a.status, left0 + (p - (lo - T)), a.ring_len)))
            v[e] = l_intra ? lloc[p - (lo - T)] : ld_cg(left + (p - (lo - T)));
        }
      }
      if (sr >= 0 && Win::touches(warp, hi, hi + T)) {
        const int64_t right0 = (static_cast<int64_t>(sr) * R + (vr & (R - 1))) * 2 * T;
        const real* right = strips + right0;
        const real* rloc = rstrip + static_cast<size_t>(vr & (R - 1)) * T;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = Win::pos(warp, lane, e);
          if (p >= hi && p < hi + T && (r_intra || index_ok(a.status, right0 + (p - hi), a.ring_len)))
            v[e] = r_intra ? rloc[p - hi] : ld_cg(right + (p - hi));
        }
      }
    }
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
    // The barrier inside also keeps sh_v stable until every thread has read it.
    publish_strips<real, E, Win>(v, strips, my_prog, out, s, R, T, lo, hi, j + 1, stalled, warp, lane, nwarps, tid,
                                 a.status, a.ring_len);
  }

  if (ok) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = Win::pos(warp, lane, e);
      if (p >= lo && p < hi && Win::owner(warp, lane, e, nwarps) && index_ok(a.status, a0 + (p - lo), N))
        uout[a0 + (p - lo)] = v[e];
    }
  }
  // Every thread of the cluster reaches this point (all waits are bounded),
  // so no CTA leaves while a neighbour may still write into its strips.
  if (C > 1) cluster_sync_all();
}

// Dynamic shared memory of a cluster launch: the two strip rings.
inline size_t cluster_strip_bytes(int elem_bytes, int R, int T) { return 2 * static_cast<size_t>(R) * T * elem_bytes; }

template <typename real, int E>
int launch_t(const SegmentRun& a, int threads, cudaStream_t st) {
  SegmentRun args = a;
  set_run_params(args);
  if (a.cluster > 1) {
    // A cluster launch (not cooperative): the residency of every cluster was
    // checked by blocked_cluster_size, and every wait in the kernel is
    // bounded, so a CTA that could not be scheduled makes the run time out.
    const size_t smem = cluster_strip_bytes(sizeof(real), a.R, a.T);
    if (cudaFuncSetAttribute(async_blocked_kernel<real, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return HEAT1D_ERR_CUDA;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_launch_config(a.S, threads, smem, a.cluster, st, attr);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, async_blocked_kernel<real, E>, args);
    return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
  }
  void* params[] = {&args};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(async_blocked_kernel<real, E>), dim3(a.S),
                                              dim3(threads), params, 0, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

template <typename real, int E>
int cluster_size_t(int threads, int S, int R, int T, int wanted) {
  const size_t smem = cluster_strip_bytes(sizeof(real), R, T);
  if (smem > kMaxClusterStripBytes) return wanted > 1 ? 0 : 1;
  if (cudaFuncSetAttribute(async_blocked_kernel<real, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess) {
    cudaGetLastError();
    return wanted > 1 ? 0 : 1;
  }
  return pick_cluster_size(async_blocked_kernel<real, E>, S, threads, smem, wanted);
}

}  // namespace

int blocked_cluster_size(int dtype, int E, int threads, int S, int R, int T, int wanted) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 2: return f64 ? cluster_size_t<double, 2>(threads, S, R, T, wanted) : cluster_size_t<float, 2>(threads, S, R, T, wanted);
    case 4: return f64 ? cluster_size_t<double, 4>(threads, S, R, T, wanted) : cluster_size_t<float, 4>(threads, S, R, T, wanted);
    case 8: return f64 ? cluster_size_t<double, 8>(threads, S, R, T, wanted) : cluster_size_t<float, 8>(threads, S, R, T, wanted);
    case 16:
      return f64 ? cluster_size_t<double, 16>(threads, S, R, T, wanted) : cluster_size_t<float, 16>(threads, S, R, T, wanted);
    case 32: return f64 ? 0 : cluster_size_t<float, 32>(threads, S, R, T, wanted);
    default: return 0;
  }
}

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

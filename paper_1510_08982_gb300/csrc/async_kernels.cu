// async_kernels.cu -- the asynchronous run of Section 3, Eq. (eqn:async), and
// its exact replay, as one persistent cooperative launch with no barrier
// between CTAs.
//
// One CTA owns one segment (a PE of Fig. 1).  Its compute warps hold the
// segment plus one halo point per side in registers and step with no
// asynchrony inside the CTA (Section 3).  Three extra warps per CTA are the
// "network": one publishes the segment's two edge values of every version to
// global rings (release store of the segment's version counter), one per
// neighbour copies that neighbour's published versions into a ring in shared
// memory (the buffer of Section 3 that keeps the q most recent values
// received).  Separate warps let the publish fence and the two neighbours'
// L2 round trips overlap.
//
// At step k the compute warp holding a halo takes, from that local buffer,
// the newest neighbour version v <= k; it waits only while v < k-q+1 (bounded
// delay, k* in {k, ..., k-q+1}).  It records d = k - v for the trace.  In
// replay mode it waits for, and takes, exactly v = k - min(d, k) from the
// given trace.  Only the two edge warps (halo reads, edge hand-offs) stop
// after every step; the other compute warps advance each run of refresh steps
// at once, and all meet at the warp-halo refresh.
//
// Flow control: a segment cannot start step k until both neighbours have
// published version k-q+1, so no two neighbours drift more than q steps
// apart, and a ring of R >= 2q versions is never overwritten while a reader
// may still need the slot.
#include <algorithm>

#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

template <typename real, int E>
struct AsyncShared {
  WindowShared<real, async_window_halo(sizeof(real), E)> win;
  real lring[kMaxRing];  // left neighbour's right-edge values, version v at v & (R-1)
  real rring[kMaxRing];  // right neighbour's left-edge values
  real own_l[kMaxRing];  // this segment's first point per version, for the comm warp
  real own_r[kMaxRing];  // this segment's last point per version
  int lavail, ravail;    // newest neighbour version held in lring / rring (-1: none)
  int own_l_ver, own_r_ver;  // newest own version handed to the comm warp
  int compute_done;          // 1: finished, 2: aborted
};



// v[idx] for a run-time idx, by a tree of selects on the bits of idx (no
// local-memory array, log2(E) levels).
template <typename real, int E>
__device__ __forceinline__ real pick_slot(const real (&v)[E], int idx) {
  real t[E];
#pragma unroll
  for (int e = 0; e < E; ++e) t[e] = v[e];
#pragma unroll
  for (int w = 1; w < E; w *= 2) {
    const bool hi = (idx & w) != 0;
#pragma unroll
    for (int e = 0; e + w < E; e += 2 * w) t[e] = hi ? t[e + w] : t[e];
  }
  return t[0];
}

// Waits for the neighbour version this step needs and returns its value.
// Returns false if the wait ran out or the run failed elsewhere.
template <typename real>
__device__ __forceinline__ bool fetch_halo(const SegmentRun& a, const int* avail, const real* ring, int k,
                                           const uint8_t* trace_in, uint8_t* trace_out, size_t tidx, int d_replay,
                                           real& value) {
  // Step k of this launch is global step k0 + k of a resumed run; no read
  // reaches before global step 0 (a delay is clamped to the global step).
  const int kb = a.k0 < a.q ? static_cast<int>(a.k0) : a.q;
  int need;
  if (trace_in) {
    if (d_replay >= a.q) {
      raise_status(a.status, HEAT1D_ERR_TRACE);
      return false;
    }
    need = k - min(d_replay, k + kb);
  } else {
    need = max(k - a.q + 1, -kb);
  }
  int V = ld_acquire_cta_shared(avail);
  if (V < need) {
    const uint64_t t0 = global_timer_ns();
    unsigned spins = 0;
    while ((V = ld_acquire_cta_shared(avail)) < need) {
      if ((++spins & 63u) == 0) {
        if (status_failed(a.status)) return false;
        if (static_cast<int64_t>(global_timer_ns() - t0) > a.spin_limit_ns) {
          raise_status(a.status, HEAT1D_ERR_TIMEOUT);
          return false;
        }
      }
    }
  }
  const int vsel = trace_in ? need : min(V, k);
  value = ring[vsel & (a.R - 1)];
  if (trace_out) trace_out[tidx] = static_cast<uint8_t>(k - vsel);
  return true;
}

// The three communication warps (one thread each does the work).

// Publisher: pushes every new version of the segment's two edge values to its
// global rings, then release-stores the segment's version counter.
template <typename real, int E>
__device__ void publish_loop(const SegmentRun& a, AsyncShared<real, E>& sh, int s) {
  const int R = a.R;
  const int K = static_cast<int>(a.K);
  real* rings = static_cast<real*>(a.rings);
  real* my_l = rings + (static_cast<size_t>(s) * 2 + 0) * R;
  real* my_r = rings + (static_cast<size_t>(s) * 2 + 1) * R;
  int* my_prog = a.prog + static_cast<size_t>(s) * kProgStride;
  const bool stalled = s == a.stall_segment;
  const bool replay = a.trace_in != nullptr;
  int pub = -1;
  uint64_t t_idle = global_timer_ns();
  unsigned spins = 0;
  while (true) {
    const int w = min(ld_acquire_cta_shared(&sh.own_l_ver), ld_acquire_cta_shared(&sh.own_r_ver));
    if (!stalled && w > pub) {
      for (int x = max(pub + 1, w - R + 1); x <= w; ++x) {
        const int j = x & (R - 1);
        st_cg(my_l + j, sh.own_l[j]);
        st_cg(my_r + j, sh.own_r[j]);
      }
      st_release_gpu(my_prog, w);
      pub = w;
      t_idle = global_timer_ns();
      continue;
    }
    const int done = ld_acquire_cta_shared(&sh.compute_done);
    if (done == 2 || (done == 1 && (pub >= K || stalled))) break;
    // Back off between polls: a tight shared-memory spin takes issue and
    // shared-memory slots from the compute warps.  A replay waits on exact
    // versions, so its publisher naps less (measured on the 2^20-point rod:
    // free runs are fastest at 256 ns, replays at 64 ns).
    __nanosleep(replay ? 64 : 256);
    if ((++spins & 63u) == 0) {
      if (status_failed(a.status)) break;
      if (static_cast<int64_t>(global_timer_ns() - t_idle) > a.spin_limit_ns) {
        raise_status(a.status, HEAT1D_ERR_TIMEOUT);
        break;
      }
    }
  }
}

// Puller (a whole warp): copies each new version of one neighbour's facing
// edge value from its global ring into the local ring, then release-stores
// the newest version held (the buffer of Section 3 that keeps the most recent
// received values).  Lane 0 acquires the neighbour's version counter; after a
// warp barrier (which orders that acquire before the other lanes' loads) the
// lanes copy the new versions in parallel, so one pass costs two L2 round
// trips however many versions arrived.
template <typename real, int E>
__device__ void pull_loop(const SegmentRun& a, AsyncShared<real, E>& sh, const int* nprog, const real* nring,
                          real* lring, int* avail, int lane, const real* nhist) {
  const int R = a.R;
  int seen = -1;
  if (nhist) {
    // A resumed run: the neighbour's edge value at the last q steps before
    // this launch (versions -q+1 .. 0) is already known.
    for (int j = lane; j < a.q; j += 32) lring[(j - a.q + 1) & (R - 1)] = nhist[j];
    __syncwarp();
    if (lane == 0) st_release_cta_shared(avail, 0);
    seen = 0;
  }
  uint64_t t_idle = global_timer_ns();
  unsigned spins = 0;
  while (true) {
    int P = 0;
    if (lane == 0) P = ld_acquire_gpu(nprog);
    __syncwarp();
    P = __shfl_sync(kFullMask, P, 0);
    if (P > seen) {
      for (int x = max(seen + 1, P - R + 1) + lane; x <= P; x += 32) lring[x & (R - 1)] = ld_cg(nring + (x & (R - 1)));
      __syncwarp();
      if (lane == 0) st_release_cta_shared(avail, P);
      seen = P;
      t_idle = global_timer_ns();
      continue;
    }
    int stop = 0;
    if (lane == 0) {
      if (ld_acquire_cta_shared(&sh.compute_done)) {
        stop = 1;  // no more reads needed
      } else if ((++spins & 63u) == 0) {
        if (status_failed(a.status)) {
          stop = 1;
        } else if (static_cast<int64_t>(global_timer_ns() - t_idle) > a.spin_limit_ns) {
          raise_status(a.status, HEAT1D_ERR_TIMEOUT);
          stop = 1;
        }
      }
    }
    if (__shfl_sync(kFullMask, stop, 0)) break;
  }
}

template <typename real, int E>
__global__ void __launch_bounds__(max_async_threads(sizeof(real), E), 1) async_persistent_kernel(SegmentRun a) {
  using Win = Window<E, async_window_halo(sizeof(real), E)>;
  constexpr int kRefresh = Win::H;  // steps between two halo refreshes
  __shared__ AsyncShared<real, E> sh;
  const int s = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwc = (blockDim.x >> 5) - kCommWarps;  // compute warps; the last three communicate
  const unsigned nthreads_c = static_cast<unsigned>(nwc) * 32u;
  if (tid == 0) {
    sh.lavail = -1;
    sh.ravail = -1;
    sh.own_l_ver = -1;
    sh.own_r_ver = -1;
    sh.compute_done = 0;
  }
  __syncthreads();

  if (warp >= nwc) {
    real* rings = static_cast<real*>(a.rings);
    const int sl = s > 0 ? s - 1 : (a.periodic ? a.S - 1 : -1);  // neighbours (ring when periodic)
    const int sr = s + 1 < a.S ? s + 1 : (a.periodic ? 0 : -1);
    if (warp == nwc) {
      if (lane == 0) publish_loop<real, E>(a, sh, s);
    } else {
      // warp nwc+1 pulls the left neighbour's right edge, warp nwc+2 the
      // right neighbour's left edge
      const bool from_left = warp == nwc + 1;
      const int nb = from_left ? sl : sr;
      // history layout [S][2][q]: side 0 the first point, side 1 the last point
      const real* nhist = (nb >= 0 && a.hist_in)
                              ? static_cast<const real*>(a.hist_in) + (static_cast<size_t>(nb) * 2 + (from_left ? 1 : 0)) * a.q
                              : nullptr;
      if (nb >= 0)
        pull_loop<real, E>(a, sh, a.prog + static_cast<size_t>(nb) * kProgStride,
                           rings + (static_cast<size_t>(nb) * 2 + (from_left ? 1 : 0)) * a.R,
                           from_left ? sh.lring : sh.rring, from_left ? &sh.lavail : &sh.ravail, lane, nhist);
    }
    return;
  }

  const int64_t N = a.N;
  const int64_t a0 = a.seg_off[s];
  const int L = static_cast<int>(a.seg_off[s + 1] - a0);
  const int K = static_cast<int>(a.K);
  const int S = a.S;
  const real c1 = kparam<real>(a.c1, a.c1_f), cN = kparam<real>(a.cN, a.cN_f);
  const Coef<real> coef{kparam<real>(a.r, a.r_f), kparam<real>(a.one, a.one_f)};  // one = 1 at run time
  const real* __restrict__ uin = static_cast<const real*>(a.u_in);
  real* __restrict__ uout = static_cast<real*>(a.u_out);
  const bool periodic = a.periodic != 0;
  const bool has_left = s > 0 || periodic, has_right = s + 1 < S || periodic;

  // Position p holds global point a0 - 1 + p: positions 0 and L+1 are the
  // halos, written from the neighbours' versions before every step.  The
  // Dirichlet ends are points end_lo and end_hi; on the periodic ring they are
  // moved out of reach (every point is updated).
  const int64_t end_lo = periodic ? -2 : 0, end_hi = periodic ? N + 1 : N - 1;
  real v[E];
  unsigned fixed = 0;
  int e_first = -1, e_last = -1, e_rh = -1;  // slots of this thread holding positions 1, L (owners) and L+1
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = Win::pos(warp, lane, e);
    const int64_t g = a0 - 1 + p;
    real x = static_cast<real>(0);
    if (p >= 1 && p <= L) x = uin[g];
    if (g == end_lo) x = c1;
    if (g == end_hi) x = cN;
    v[e] = x;
    // Only points outside the rod and the Dirichlet ends are held.  The halo
    // positions 0 and L+1 are written before every step that reads them, and
    // positions past L+1 reach no point of the segment, so those warps can
    // step without the per-point selects of the masked mode.
    if (g <= end_lo || g >= end_hi) fixed |= 1u << e;
    const bool own = Win::owner(warp, lane, e, nwc);
    if (p == 1 && own) e_first = e;
    if (p == L && own) e_last = e;
    // the copy of position L+1 in the same warp as position L's owner
    if (p == L + 1 && ((e > 0 && Win::owner(warp, lane, e - 1, nwc)) ||
                       (e == 0 && lane > 0 && Win::owner(warp, lane - 1, E - 1, nwc))))
      e_rh = e;
  }
  const int mode = tile_mode<E>(fixed);
  real* snap = static_cast<real*>(a.snap);
  if (snap) {  // row 0: the state at step 0
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = Win::pos(warp, lane, e);
      if (p >= 1 && p <= L && Win::owner(warp, lane, e, nwc)) snap[a0 - 1 + p] = v[e];
    }
  }
  const bool left_reader = has_left && warp == 0 && lane == 0;  // position 0 is (warp 0, lane 0, slot 0)
  const bool right_reader = has_right && e_rh >= 0;

  // Version 0 of the edges goes to the comm warp.
  if (e_first >= 0) {
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e == e_first) sh.own_l[0] = v[e];
    st_release_cta_shared(&sh.own_l_ver, 0);
  }
  if (e_last >= 0) {
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e == e_last) sh.own_r[0] = v[e];
    st_release_cta_shared(&sh.own_r_ver, 0);
  }

  const uint8_t* trace_in = a.trace_in;
  uint8_t* trace_out = a.trace_out;
  // S-1 boundaries (S on the periodic ring, boundary b joining b and b+1 mod S)
  const size_t tstride = static_cast<size_t>(periodic ? S : S - 1) * 2;
  const size_t tl = has_left ? static_cast<size_t>((s + S - 1) % S) * 2 + 1 : 0;  // side 1 of boundary s-1
  const size_t tr = static_cast<size_t>(s) * 2 + 0;                               // side 0 of boundary s
  int dl_next = 0, dr_next = 0;
  if (trace_in && K > 0) {
    if (left_reader) dl_next = __ldg(trace_in + tl);
    if (right_reader) dr_next = __ldg(trace_in + tr);
  }

  // Only the warps that read a halo or hand an edge to the publisher need to
  // stop after every step.  The others advance each run of kRefresh steps
  // with the two-array step (no per-step checks, no register rotation); the
  // arithmetic is the same.  While snapshots are recorded every warp steps
  // one at a time, so that it can store the state of any step.
  const bool edge_warp = __any_sync(kFullMask, left_reader || right_reader || e_first >= 0 || e_last >= 0);
  const bool per_step = edge_warp || snap != nullptr;
  bool failed = false;   // a wait of this thread gave up: no more waits until the CTA leaves
  bool aborted = false;
  int parity = 0;
  for (int k0 = 0; k0 < K; k0 += kRefresh) {
    const int n = min(kRefresh, K - k0);
    if (!per_step) {
      if (mode == kTileFree)
        warp_run<real, E, kTileFree, kRefresh>(v, fixed, coef, n);
      else if (mode == kTileEnds)
        warp_run<real, E, kTileEnds, kRefresh>(v, fixed, coef, n);
      else if (mode == kTileMasked)
        warp_run<real, E, kTileMasked, kRefresh>(v, fixed, coef, n);
    } else {
      // One step from `in` to `out`: the halo reads before it, the state
      // records and edge hand-offs after it.  Steps alternate between v and
      // w, so the loop carries no register rotation.
      auto edge_step = [&](real (&in)[E], real (&out)[E], int k) {
        if (left_reader && !failed) {
          const int d = dl_next;
          if (trace_in && k + 1 < K) dl_next = __ldg(trace_in + static_cast<size_t>(k + 1) * tstride + tl);
          real val;
          if (fetch_halo<real>(a, &sh.lavail, sh.lring, k, trace_in, trace_out, static_cast<size_t>(k) * tstride + tl,
                               d, val))
            in[0] = val;
          else
            failed = true;
        }
        if (right_reader && !failed) {
          const int d = dr_next;
          if (trace_in && k + 1 < K) dr_next = __ldg(trace_in + static_cast<size_t>(k + 1) * tstride + tr);
          real val;
          if (fetch_halo<real>(a, &sh.ravail, sh.rring, k, trace_in, trace_out, static_cast<size_t>(k) * tstride + tr,
                               d, val)) {
#pragma unroll
            for (int e = 0; e < E; ++e)
              if (e == e_rh) in[e] = val;
          } else {
            failed = true;
          }
        }
        if (mode == kTileFree) {
          warp_step_to<real, E, kTileFree>(in, out, fixed, coef);
        } else if (mode == kTileEnds) {
          warp_step_to<real, E, kTileEnds>(in, out, fixed, coef);
        } else if (mode == kTileMasked) {
          warp_step_to<real, E, kTileMasked>(in, out, fixed, coef);
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) out[e] = in[e];
        }
        const int ver = k + 1, j = ver & (a.R - 1);
        if (snap && ver % a.snap_every == 0) {  // owners record the state at step ver
          real* row = snap + static_cast<size_t>(ver / a.snap_every) * N;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int p = Win::pos(warp, lane, e);
            if (p >= 1 && p <= L && Win::owner(warp, lane, e, nwc)) row[a0 - 1 + p] = out[e];
          }
        }
        if (e_first >= 0) {  // position 1: always slot 1 of lane 0 in warp 0
          sh.own_l[j] = out[1];
          st_release_cta_shared(&sh.own_l_ver, ver);
        }
        if (e_last >= 0) {
          sh.own_r[j] = pick_slot<real, E>(out, e_last);
          st_release_cta_shared(&sh.own_r_ver, ver);
        }
      };
      real w[E];
      int k = k0;
      for (; k + 1 < k0 + n; k += 2) {
        edge_step(v, w, k);
        edge_step(w, v, k + 1);
      }
      if (k < k0 + n) {
        edge_step(v, w, k);
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = w[e];
      }
    }
    // Refresh the warp halos after every run of kRefresh steps (and after the
    // last step); the refresh barrier also tells every warp whether a wait
    // gave up.
    const bool any_failed = warp_refresh<real, E, Win::H>(v, sh.win, parity, warp, lane, nwc, nthreads_c, failed);
    parity ^= 1;
    if (any_failed) {
      aborted = true;
      break;
    }
  }

#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = Win::pos(warp, lane, e);
    if (p >= 1 && p <= L && Win::owner(warp, lane, e, nwc)) uout[a0 - 1 + p] = v[e];
  }
  // The edge values of the last q steps, for a later resumed run: versions
  // K-q+1 .. K of this launch from the hand-off rings (written by these same
  // threads), older ones from the history this launch started from.
  if (a.hist_out && !aborted && (e_first >= 0 || e_last >= 0)) {
    real* ho = static_cast<real*>(a.hist_out);
    const real* hi_ = static_cast<const real*>(a.hist_in);
    for (int j = 0; j < a.q; ++j) {
      const int ver = K - a.q + 1 + j;
      if (e_first >= 0) {
        const real x = ver >= 0 ? sh.own_l[ver & (a.R - 1)]
                                : (hi_ ? hi_[(static_cast<size_t>(s) * 2 + 0) * a.q + (ver + a.q - 1)] : sh.own_l[0]);
        ho[(static_cast<size_t>(s) * 2 + 0) * a.q + j] = x;
      }
      if (e_last >= 0) {
        const real x = ver >= 0 ? sh.own_r[ver & (a.R - 1)]
                                : (hi_ ? hi_[(static_cast<size_t>(s) * 2 + 1) * a.q + (ver + a.q - 1)] : sh.own_r[0]);
        ho[(static_cast<size_t>(s) * 2 + 1) * a.q + j] = x;
      }
    }
  }
  named_barrier_sync(1, nthreads_c);
  if (tid == 0) st_release_cta_shared(&sh.compute_done, aborted ? 2 : 1);
}

template <typename real, int E>
int launch_async_t(const SegmentRun& a, int threads, cudaStream_t st) {
  SegmentRun args = a;
  set_run_params(args);
  void* params[] = {&args};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(async_persistent_kernel<real, E>), dim3(a.S),
                                              dim3(threads + 32 * kCommWarps), params, 0, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

template <typename real, int E>
int resident_t(int threads) {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, async_persistent_kernel<real, E>, threads + 32 * kCommWarps, 0) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace

int launch_async_persistent(const SegmentRun& a, int dtype, int E, int threads, cudaStream_t st) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 2: return f64 ? launch_async_t<double, 2>(a, threads, st) : launch_async_t<float, 2>(a, threads, st);
    case 4: return f64 ? launch_async_t<double, 4>(a, threads, st) : launch_async_t<float, 4>(a, threads, st);
    case 8: return f64 ? launch_async_t<double, 8>(a, threads, st) : launch_async_t<float, 8>(a, threads, st);
    case 16: return f64 ? launch_async_t<double, 16>(a, threads, st) : launch_async_t<float, 16>(a, threads, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

int max_resident_async(int dtype, int E, int threads) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 2: return f64 ? resident_t<double, 2>(threads) : resident_t<float, 2>(threads);
    case 4: return f64 ? resident_t<double, 4>(threads) : resident_t<float, 4>(threads);
    case 8: return f64 ? resident_t<double, 8>(threads) : resident_t<float, 8>(threads);
    case 16: return f64 ? resident_t<double, 16>(threads) : resident_t<float, 16>(threads);
    default: return 0;
  }
}

}  // namespace heat1d_impl

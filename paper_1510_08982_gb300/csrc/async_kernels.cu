// async_kernels.cu -- the asynchronous run of Section 3, Eq. (eqn:async), and
// its exact replay, as one persistent launch with no barrier between CTAs.
//
// One CTA owns one segment (a PE of Fig. 1).  Its compute warps hold the
// segment plus one halo point per side in registers and step with no
// asynchrony inside the CTA (Section 3).
//
// Tagged slots.  Every edge value travels with its version: each 32-bit half
// of the value shares a 64-bit word with the version number, so a reader that
// finds the version it wants in every word of a slot holds that version's
// value.  A slot caught in the middle of an update simply does not match yet;
// no release/acquire pair, no fence and no version counter sit on the path.
// The thread that computes a segment's first (last) point writes each new
// version into the ring of R slots that its left (right) neighbour reads:
//  - a neighbour in the same thread-block cluster: straight into that CTA's
//    shared-memory ring (distributed shared memory);
//  - any other neighbour: into the segment's ring in global memory, which a
//    puller warp of the neighbour mirrors into its own shared-memory ring.
// The shared-memory ring is the buffer of Section 3 that keeps the most
// recent values received.
//
// At step k the compute thread holding a halo takes, from its shared ring,
// the newest neighbour version v <= k; it waits only while no v >= k-q+1 is
// there (bounded delay, k* in {k, ..., k-q+1}), and records d = k - v for the
// trace.  In replay mode it waits for, and takes, exactly v = k - min(d, k).
// Only the two edge warps stop after every step; the other compute warps
// advance each run of refresh steps at once, and all meet at the warp-halo
// refresh.
//
// Flow control and ring safety: a segment cannot start step k until both
// neighbours have produced version k-q+1, so neighbours drift at most q-1
// steps apart and a writer overwrites the slot of version v only once its
// reader needs versions above v (R >= 2q).  The reader's own loads come
// first: the value it hands on at version k+1 is computed (its edge point's
// update) from the halo it read at step k, so no neighbour can see that
// version before those reads are done.
#include <algorithm>

#include "checked.cuh"
#include "cluster.cuh"
#include "common.cuh"
#include "impl.h"
#include "slots.cuh"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

template <typename real, int E>
struct AsyncShared {
  WindowShared<real, async_window_halo(sizeof(real), E)> win;
  // Tagged slots [R][W]: version v at slot v & (R-1).
  unsigned long long lin[kMaxRing * Tag<real>::W];  // the left neighbour's last point
  unsigned long long rin[kMaxRing * Tag<real>::W];  // the right neighbour's first point
  real own_l[kMaxRing];  // this segment's first point per version (for the edge history)
  real own_r[kMaxRing];  // this segment's last point per version
  unsigned long long dst[2];  // where the first [0] and last [1] points go (see hand_off)
  int compute_done;      // 1: finished, 2: aborted
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

// Version v of a ring in this CTA's shared memory, if every word of its slot
// carries v.
template <typename real>
__device__ __forceinline__ bool read_slot(const unsigned long long* ring, int R, int v, real& x) {
  constexpr int W = Tag<real>::W;
  const unsigned long long* p = ring + static_cast<size_t>(v & (R - 1)) * W;
  uint32_t b[W];
  bool ok = true;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const unsigned long long u = ld_slot_shared(p + w);
    ok = ok && slot_ver(u) == v;
    b[w] = static_cast<uint32_t>(u);
  }
  if (ok) x = Tag<real>::join(b);
  return ok;
}

// Waits for the neighbour version this step reads and returns its value.
// Returns false if the wait ran out or the run failed elsewhere.
template <typename real>
__device__ __forceinline__ bool fetch_halo(const SegmentRun& a, const unsigned long long* ring, int k, bool replay,
                                           uint8_t* trace_out, size_t tidx, int d_replay, real& value) {
  // Step k of this launch is global step k0 + k of a resumed run; no read
  // reaches before global step 0 (a delay is clamped to the global step).
  const int kb = a.k0 < a.q ? static_cast<int>(a.k0) : a.q;
  int lo, hi;  // versions this step may take; the newest present wins
  if (replay) {
    if (d_replay >= a.q) {
      raise_status(a.status, HEAT1D_ERR_TRACE);
      return false;
    }
    lo = hi = k - min(d_replay, k + kb);
  } else {
    hi = k;
    lo = max(k - a.q + 1, -kb);
  }
  uint64_t t0 = 0;
  unsigned spins = 0;
  int v;
  while (true) {
    for (v = hi; v >= lo; --v)
      if (read_slot<real>(ring, a.R, v, value)) break;
    if (v >= lo) break;
    if (spins == 0) t0 = global_timer_ns();
    if ((++spins & 63u) == 0) {
      if (status_failed(a.status)) return false;
      if (static_cast<int64_t>(global_timer_ns() - t0) > a.spin_limit_ns) {
        raise_status(a.status, HEAT1D_ERR_TIMEOUT);
        return false;
      }
    }
  }
  if (trace_out && index_ok(a.status, static_cast<int64_t>(tidx), a.trace_len))
    trace_out[tidx] = static_cast<uint8_t>(k - v);
  return true;
}

// Puller (a whole warp): mirrors a neighbour's ring in global memory into
// this CTA's shared ring.  Lane l looks after slots l, l+32, ...; a slot is
// copied when all its words carry one version newer than the one held.
template <typename real>
__device__ void pull_loop(const SegmentRun& a, const int* compute_done, const unsigned long long* g,
                          unsigned long long* loc, int lane) {
  constexpr int W = Tag<real>::W;
  const int R = a.R;
  uint64_t t_idle = global_timer_ns();
  unsigned spins = 0;
  while (true) {
    bool moved = false;
    for (int j = lane; j < R; j += 32) {
      unsigned long long w[W];
#pragma unroll
      for (int x = 0; x < W; ++x) w[x] = ld_slot_global(g + static_cast<size_t>(j) * W + x);
      const int v = slot_ver(w[0]);
      bool same = true;
#pragma unroll
      for (int x = 1; x < W; ++x) same = same && slot_ver(w[x]) == v;
      if (same && v > slot_ver(ld_slot_shared(loc + static_cast<size_t>(j) * W))) {
#pragma unroll
        for (int x = 0; x < W; ++x) st_slot_shared(loc + static_cast<size_t>(j) * W + x, w[x]);
        moved = true;
      }
    }
    if (__any_sync(kFullMask, moved)) {
      t_idle = global_timer_ns();
      continue;
    }
    int stop = 0;
    if (lane == 0) {
      if (ld_acquire_cta_shared(compute_done)) {
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

// Where one edge value of this segment goes, as one word: bit 63 set and the
// neighbour's shared ring address (mapa) in the low half for a neighbour in
// the cluster; else the address of this segment's ring in global memory; 0
// for nowhere (no neighbour on that side, or a stalled segment).  Kept in
// shared memory: the edge threads read it once per step, off their
// registers.
constexpr unsigned long long kRemoteDst = 1ull << 63;

template <typename real>
__device__ __forceinline__ void hand_off(unsigned long long dst, int R, int ver, real x) {
  constexpr int W = Tag<real>::W;
  if (!dst) return;
  uint32_t b[W];
  Tag<real>::split(x, b);
  const int j = ver & (R - 1);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const unsigned long long u = slot_word(ver, b[w]);
    if (dst & kRemoteDst)
      st_slot_cluster(static_cast<uint32_t>(dst) + static_cast<uint32_t>((j * W + w) * sizeof(unsigned long long)), u);
    else
      st_slot_global(reinterpret_cast<unsigned long long*>(dst) + static_cast<size_t>(j) * W + w, u);
  }
}

template <typename real, int E>
__global__ void __launch_bounds__(max_async_threads(sizeof(real), E), 1) async_persistent_kernel(SegmentRun a) {
  using Win = Window<E, async_window_halo(sizeof(real), E)>;
  constexpr int kRefresh = Win::H;  // steps between two halo refreshes
  constexpr int W = Tag<real>::W;
  __shared__ AsyncShared<real, E> sh;
  const int s = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwc = (blockDim.x >> 5) - kCommWarps;  // compute warps; the last two pull
  const unsigned nthreads_c = static_cast<unsigned>(nwc) * 32u;
  const int R = a.R;
  const int sl = s > 0 ? s - 1 : (a.periodic ? a.S - 1 : -1);  // neighbours (ring when periodic)
  const int sr = s + 1 < a.S ? s + 1 : (a.periodic ? 0 : -1);
  // Neighbours in this CTA's cluster: a 1-D grid in clusters of C consecutive
  // CTAs (rank = s mod C); on the periodic ring the two ends only when one
  // cluster holds every segment.
  const int C = a.cluster;
  const unsigned rank = C > 1 ? cluster_rank() : 0u;
  const bool l_intra = C > 1 && sl >= 0 && (rank > 0 || C == a.S);
  const bool r_intra = C > 1 && sr >= 0 && (static_cast<int>(rank) + 1 < C || C == a.S);
  unsigned long long* rings = static_cast<unsigned long long*>(a.rings);  // [S][2][R][W]: side 0 first point, 1 last

  for (int i = tid; i < R * W; i += blockDim.x) {
    sh.lin[i] = kEmptySlot;
    sh.rin[i] = kEmptySlot;
  }
  if (tid == 0) sh.compute_done = 0;
  __syncthreads();
  if (a.hist_in) {
    // A resumed run: the neighbours' edge values at the last q steps before
    // this launch (versions -q+1 .. 0).  History layout [S][2][q]: side 0 a
    // segment's first point, side 1 its last point, oldest first.
    const real* hist = static_cast<const real*>(a.hist_in);
    for (int i = tid; i < 2 * a.q; i += blockDim.x) {
      const bool left = i < a.q;
      const int j = left ? i : i - a.q;
      const int nb = left ? sl : sr;
      if (nb < 0) continue;
      const int ver = j - a.q + 1;
      const int64_t hi_idx = (static_cast<int64_t>(nb) * 2 + (left ? 1 : 0)) * a.q + j;
      if (!index_ok(a.status, hi_idx, a.hist_len)) continue;
      uint32_t b[W];
      Tag<real>::split(hist[hi_idx], b);
      unsigned long long* ring = left ? sh.lin : sh.rin;
#pragma unroll
      for (int w = 0; w < W; ++w) ring[(ver & (R - 1)) * W + w] = slot_word(ver, b[w]);
    }
  }
  __syncthreads();
  // No CTA of the cluster may write into a neighbour before that neighbour
  // has cleared its rings.
  if (C > 1) cluster_sync_all();

  if (warp >= nwc) {
    // warp nwc mirrors the left neighbour's last point, warp nwc+1 the right
    // neighbour's first point (unless that neighbour is in the cluster and
    // writes here itself)
    const bool from_left = warp == nwc;
    const int nb = from_left ? sl : sr;
    const int64_t ring0 = (static_cast<int64_t>(nb) * 2 + (from_left ? 1 : 0)) * R * W;
    if (nb >= 0 && !(from_left ? l_intra : r_intra) && index_ok(a.status, ring0 + R * W - 1, a.ring_len))
      pull_loop<real>(a, &sh.compute_done, rings + ring0, from_left ? sh.lin : sh.rin, lane);
  } else {
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
    // Dirichlet ends are points end_lo and end_hi; on the periodic ring they
    // are moved out of reach (every point is updated).
    const int64_t end_lo = periodic ? -2 : 0, end_hi = periodic ? N + 1 : N - 1;
    real v[E];
    unsigned fixed = 0;
    int e_first = -1, e_last = -1, e_rh = -1;  // slots of this thread holding positions 1, L (owners) and L+1
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = Win::pos(warp, lane, e);
      const int64_t g = a0 - 1 + p;
      real x = static_cast<real>(0);
      if (p >= 1 && p <= L && index_ok(a.status, g, N)) x = uin[g];
      if (g == end_lo) x = c1;
      if (g == end_hi) x = cN;
      v[e] = x;
      // Only points outside the rod and the Dirichlet ends are held.  The
      // halo positions 0 and L+1 are written before every step that reads
      // them, and positions past L+1 reach no point of the segment, so those
      // warps can step without the per-point selects of the masked mode.
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
        if (p >= 1 && p <= L && Win::owner(warp, lane, e, nwc) && index_ok(a.status, a0 - 1 + p, a.snap_len))
          snap[a0 - 1 + p] = v[e];
      }
    }
    const bool left_reader = has_left && warp == 0 && lane == 0;  // position 0 is (warp 0, lane 0, slot 0)
    const bool right_reader = has_right && e_rh >= 0;

    // Where this segment's first and last points go (a stalled segment hands
    // nothing on): the left neighbour reads the first point, the right one
    // the last.
    const bool stalled = s == a.stall_segment;
    if (e_first >= 0) {
      unsigned long long d = 0;
      // (a ring in global memory must lie wholly inside the rings buffer)
      if (!stalled && sl >= 0 && (l_intra || index_ok(a.status, (static_cast<int64_t>(s) * 2 + 1) * R * W - 1, a.ring_len)))
        d = l_intra ? kRemoteDst | cluster_addr(sh.rin, rank == 0 ? static_cast<unsigned>(C - 1) : rank - 1)
                    : reinterpret_cast<unsigned long long>(rings + (static_cast<size_t>(s) * 2 + 0) * R * W);
      sh.dst[0] = d;
    }
    if (e_last >= 0) {
      unsigned long long d = 0;
      if (!stalled && sr >= 0 && (r_intra || index_ok(a.status, (static_cast<int64_t>(s) * 2 + 2) * R * W - 1, a.ring_len)))
        d = r_intra ? kRemoteDst | cluster_addr(sh.lin, static_cast<int>(rank) + 1 == C ? 0u : rank + 1)
                    : reinterpret_cast<unsigned long long>(rings + (static_cast<size_t>(s) * 2 + 1) * R * W);
      sh.dst[1] = d;
    }

    // Version 0 of the edges (the state the run starts from).
    if (e_first >= 0) {
      real x = v[0];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e == e_first) x = v[e];
      sh.own_l[0] = x;
      hand_off<real>(sh.dst[0], R, 0, x);
    }
    if (e_last >= 0) {
      real x = v[0];
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (e == e_last) x = v[e];
      sh.own_r[0] = x;
      hand_off<real>(sh.dst[1], R, 0, x);
    }

    const uint8_t* trace_in = a.trace_in;
    uint8_t* trace_out = a.trace_out;
    const bool replay = trace_in != nullptr;
    // S-1 boundaries (S on the periodic ring, boundary b joining b and b+1 mod S)
    const int tstride = (periodic ? S : S - 1) * 2;
    const int tl = has_left ? ((s + S - 1) % S) * 2 + 1 : 0;  // side 1 of boundary s-1
    const int tr = s * 2 + 0;                                 // side 0 of boundary s
    int dl_next = 0, dr_next = 0;
    if (replay && K > 0) {
      if (left_reader && index_ok(a.status, tl, a.trace_len)) dl_next = __ldg(trace_in + tl);
      if (right_reader && index_ok(a.status, tr, a.trace_len)) dr_next = __ldg(trace_in + tr);
    }

    // Only the warps that read a halo or hand an edge on need to stop after
    // every step.  The others advance each run of kRefresh steps with the
    // two-array step (no per-step checks, no register rotation); the
    // arithmetic is the same.  While snapshots are recorded every warp steps
    // one at a time, so that it can store the state of any step.
    const bool edge_warp = __any_sync(kFullMask, left_reader || right_reader || e_first >= 0 || e_last >= 0);
    const bool per_step = edge_warp || snap != nullptr;
    bool failed = false;  // a wait of this thread gave up: no more waits until the CTA leaves
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
            if (replay && k + 1 < K && index_ok(a.status, static_cast<int64_t>(k + 1) * tstride + tl, a.trace_len))
              dl_next = __ldg(trace_in + static_cast<size_t>(k + 1) * tstride + tl);
            real val;
            if (fetch_halo<real>(a, sh.lin, k, replay, trace_out, static_cast<size_t>(k) * tstride + tl, d, val))
              in[0] = val;
            else
              failed = true;
          }
          if (right_reader && !failed) {
            const int d = dr_next;
            if (replay && k + 1 < K && index_ok(a.status, static_cast<int64_t>(k + 1) * tstride + tr, a.trace_len))
              dr_next = __ldg(trace_in + static_cast<size_t>(k + 1) * tstride + tr);
            real val;
            if (fetch_halo<real>(a, sh.rin, k, replay, trace_out, static_cast<size_t>(k) * tstride + tr, d, val)) {
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
          const int ver = k + 1;
          if (e_first >= 0) {  // position 1: always slot 1 of lane 0 in warp 0
            hand_off<real>(sh.dst[0], R, ver, out[1]);
            sh.own_l[ver & (R - 1)] = out[1];
          }
          if (e_last >= 0) {
            const real x = pick_slot<real, E>(out, e_last);
            hand_off<real>(sh.dst[1], R, ver, x);
            sh.own_r[ver & (R - 1)] = x;
          }
          if (a.snap && ver % a.snap_every == 0) {  // owners record the state at step ver
            const int64_t row0 = static_cast<int64_t>(ver / a.snap_every) * N;
            real* row = static_cast<real*>(a.snap) + row0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int p = Win::pos(warp, lane, e);
              if (p >= 1 && p <= L && Win::owner(warp, lane, e, nwc) && index_ok(a.status, row0 + a0 - 1 + p, a.snap_len))
                row[a0 - 1 + p] = out[e];
            }
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
      // Refresh the warp halos after every run of kRefresh steps (and after
      // the last step); the refresh barrier also tells every warp whether a
      // wait gave up.
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
      if (p >= 1 && p <= L && Win::owner(warp, lane, e, nwc) && index_ok(a.status, a0 - 1 + p, N))
        uout[a0 - 1 + p] = v[e];
    }
    // The edge values of the last q steps, for a later resumed run: versions
    // K-q+1 .. K of this launch from the own rings (written by these same
    // threads), older ones from the history this launch started from.
    if (a.hist_out && !aborted && (e_first >= 0 || e_last >= 0)) {
      real* ho = static_cast<real*>(a.hist_out);
      const real* hi_ = static_cast<const real*>(a.hist_in);
      for (int j = 0; j < a.q; ++j) {
        const int ver = K - a.q + 1 + j;
        for (int side = 0; side < 2; ++side) {
          if ((side ? e_last : e_first) < 0) continue;
          const real* own = side ? sh.own_r : sh.own_l;
          const int64_t hin = (static_cast<int64_t>(s) * 2 + side) * a.q + (ver + a.q - 1);
          const int64_t hout = (static_cast<int64_t>(s) * 2 + side) * a.q + j;
          real x = own[0];
          if (ver >= 0)
            x = own[ver & (R - 1)];
          else if (hi_ && index_ok(a.status, hin, a.hist_len))
            x = hi_[hin];
          if (index_ok(a.status, hout, a.hist_len)) ho[hout] = x;
        }
      }
    }
    named_barrier_sync(1, nthreads_c);
    if (tid == 0) st_release_cta_shared(&sh.compute_done, aborted ? 2 : 1);
  }
  // Every thread of the cluster reaches this point (all waits are bounded),
  // so no CTA leaves while a neighbour may still write into its rings.
  if (C > 1) cluster_sync_all();
}

template <typename real, int E>
int launch_async_t(const SegmentRun& a, int threads, cudaStream_t st) {
  SegmentRun args = a;
  set_run_params(args);
  if (a.cluster > 1) {
    // A cluster launch (not cooperative): the residency of every cluster was
    // checked by async_cluster_size, and every wait in the kernel is bounded,
    // so a CTA that could not be scheduled makes the run time out, not hang.
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_launch_config(a.S, threads + 32 * kCommWarps, 0, a.cluster, st, attr);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, async_persistent_kernel<real, E>, args);
    return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
  }
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

int async_cluster_size(int dtype, int E, int threads, int S, int wanted) {
  const bool f64 = dtype == HEAT1D_F64;
  const int t = threads + 32 * kCommWarps;
  switch (E) {
    case 2: return f64 ? pick_cluster_size(async_persistent_kernel<double, 2>, S, t, 0, wanted)
                       : pick_cluster_size(async_persistent_kernel<float, 2>, S, t, 0, wanted);
    case 4: return f64 ? pick_cluster_size(async_persistent_kernel<double, 4>, S, t, 0, wanted)
                       : pick_cluster_size(async_persistent_kernel<float, 4>, S, t, 0, wanted);
    case 8: return f64 ? pick_cluster_size(async_persistent_kernel<double, 8>, S, t, 0, wanted)
                       : pick_cluster_size(async_persistent_kernel<float, 8>, S, t, 0, wanted);
    case 16: return f64 ? pick_cluster_size(async_persistent_kernel<double, 16>, S, t, 0, wanted)
                        : pick_cluster_size(async_persistent_kernel<float, 16>, S, t, 0, wanted);
    default: return 0;
  }
}

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

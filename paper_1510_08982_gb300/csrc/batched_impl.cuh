// batched_impl.cuh -- many rods of uneven N, r and K in one persistent
// cooperative launch (the synchronous update of Section 2, Eq. (eqn:sync),
// applied to each rod independently).
//
// The host plans work items, each one CTA's worth, in an order of decreasing
// work; every CTA takes the next item from a global counter until the queue
// is empty.  Three kinds of item:
//   - a warp batch: up to one small rod per warp (the rod fits one warp
//     window of 32*E points); each warp runs its rod alone, registers and
//     shuffles only, no synchronisation at all;
//   - a whole rod in one CTA: the overlapping warp windows of common.cuh,
//     one CTA barrier every H steps;
//   - one part of a rod too long for one CTA: the rod is split into parts
//     with T-wide overlapped halos; parts exchange their edge points through
//     global memory every T steps and wait only for their two neighbouring
//     parts (release/acquire pass counters, no grid barrier).
// The parts of a rod are consecutive in the queue and a rod never has more
// parts than there are CTAs, so every part a CTA waits for is already held
// by another CTA or will be taken next: the launch cannot deadlock.  All
// waits are bounded.  Results are bit-identical to stepping each rod alone.
#pragma once

#include <algorithm>

#include "checked.cuh"
#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

// The waiting thread naps between polls: the batch runs two or more CTAs per
// SM, and a tight spin takes issue slots from the other CTAs' compute warps.
__device__ bool wait_flag_at_least(const int* flag, int want, int* status, int64_t limit_ns) {
  if (ld_acquire_gpu(flag) >= want) return true;
  const uint64_t t0 = global_timer_ns();
  unsigned spins = 0;
  while (ld_acquire_gpu(flag) < want) {
    if ((++spins & 31u) == 0) {
      if (status_failed(status)) return false;
      if (static_cast<int64_t>(global_timer_ns() - t0) > limit_ns) {
        raise_status(status, HEAT1D_ERR_TIMEOUT);
        return false;
      }
    }
    __nanosleep(32);
  }
  return true;
}

// Asynchronous batched run: the strip version of a neighbouring part that
// block j of this part reads -- the newest one not newer than j, waiting only
// while it is more than q-1 blocks old (free run), or exactly j - d from the
// trace (replay) -- with a bounded wait on the neighbour's version counter.
// Records the delay at `tidx` (a byte of the trace).  One thread.  Returns the
// version, or -1 after raising a failure.
__device__ int part_strip_version(const BatchRun& a, const int* nb_ver, int j, int64_t tidx) {
  int need;
  if (a.async_mode == 2) {
    const int d = index_ok(a.status, tidx, a.trace_len) ? a.trace_in[tidx] : 0;
    if (d >= a.q) {
      raise_status(a.status, HEAT1D_ERR_TRACE);
      return -1;
    }
    need = j - min(d, j);
  } else {
    need = max(j - a.q + 1, 0);
  }
  int V = ld_acquire_gpu(nb_ver);
  if (V < need) {
    const uint64_t t0 = global_timer_ns();
    unsigned spins = 0;
    while ((V = ld_acquire_gpu(nb_ver)) < need) {
      if ((++spins & 31u) == 0) {
        if (status_failed(a.status)) return -1;
        if (static_cast<int64_t>(global_timer_ns() - t0) > a.spin_limit_ns) {
          raise_status(a.status, HEAT1D_ERR_TIMEOUT);
          return -1;
        }
      }
      __nanosleep(32);
    }
  }
  const int v = a.async_mode == 2 ? need : min(V, j);
  if (a.trace_out && index_ok(a.status, tidx, a.trace_len)) a.trace_out[tidx] = static_cast<uint8_t>(j - v);
  return v;
}

// A small rod advanced by one warp: positions lane*E + e.
template <typename real, int E>
__device__ void run_warp_rod(const BatchRod& rd, real* u, int lane, double one, float one_f, int* status,
                             int64_t u_len) {
  real* x = u + rd.offset;
  const int N = static_cast<int>(rd.N);
  const real c1 = kparam<real>(rd.c1, rd.c1_f), cN = kparam<real>(rd.cN, rd.cN_f);
  const Coef<real> coef{kparam<real>(rd.r, rd.r_f), kparam<real>(one, one_f)};
  real v[E];
  unsigned fixed = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = lane * E + e;
    real y = p < N && index_ok(status, rd.offset + p, u_len) ? x[p] : static_cast<real>(0);
    if (p == 0) y = c1;
    if (p == N - 1) y = cN;
    v[e] = y;
    // only the Dirichlet ends are held: positions past u_N never reach it
    if (p == 0 || p == N - 1) fixed |= 1u << e;
  }
  const int mode = tile_mode_slot<E>(fixed);
  if (mode == kTileEnds) {
    warp_steps<real, E, kTileEnds>(v, fixed, coef, rd.K);
  } else if (mode >= kTileSlot) {
    warp_steps_slot<real, E>(mode - kTileSlot, v, fixed, coef, rd.K);
  } else {
    warp_steps<real, E, kTileMasked>(v, fixed, coef, rd.K);
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = lane * E + e;
    if (p < N && index_ok(status, rd.offset + p, u_len)) x[p] = v[e];
  }
}

// The bookkeeping of the part a CTA holds (tile bounds, its neighbours'
// slots, the rod's step count and placement).  It is written once per item
// into shared memory and re-read at every exchange, so that none of it stays
// in registers across the steps of a block: the step loop, the part's tile
// and the warp refresh then have the registers to themselves (measured: with
// the bookkeeping live, the compiler re-derived lane, warp and shared
// addresses at every warp refresh, about five more instructions per step).
struct PartState {
  int lo, hi, T, slot, part, nparts;
  int64_t K, a0, offset;
};
__device__ __forceinline__ PartState load_part(const PartState& s) {
  const volatile PartState& v = s;
  PartState r;
  r.lo = v.lo;
  r.hi = v.hi;
  r.T = v.T;
  r.slot = v.slot;
  r.part = v.part;
  r.nparts = v.nparts;
  r.K = v.K;
  r.a0 = v.a0;
  r.offset = v.offset;
  return r;
}

// kAsync: the launch of an asynchronous batched run (a separate instance, so
// that the synchronous launch carries none of the asynchronous code).
template <typename real, int E, bool kAsync>
__global__ void __launch_bounds__(max_tile_threads(sizeof(real), E), 1) batched_kernel(BatchRun a) {
  using Win = Window<E, sync_window_halo(sizeof(real), E)>;
  __shared__ WindowShared<real, Win::H> sh;
  __shared__ int sh_item;
  __shared__ int sh_ok;
  __shared__ int sh_v[2];  // asynchronous parts: strip versions read by this block (-1: failed)
  __shared__ PartState sh_part;  // the part this CTA holds
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  real* u = static_cast<real*>(a.u);
  real* edges = static_cast<real*>(a.edges);
  const double one = a.one;
  const float one_f = a.one_f;
  int parity = 0;

  while (true) {
    if (tid == 0) sh_item = static_cast<int>(atomicAdd(a.counter, 1u));
    __syncthreads();
    const int64_t idx = sh_item;
    if (idx >= a.nitems) break;
    const BatchItem it = a.items[idx];

    if (it.kind == kBatchWarps) {
      if (warp < it.count)
        run_warp_rod<real, E>(a.rods[a.warp_rods[it.rod + warp]], u, lane, one, one_f, a.status, a.u_len);
    } else if (it.kind == kBatchRod) {
      // The whole rod in this CTA; its ends are fixed, so nothing degrades.
      const BatchRod rd = a.rods[it.rod];
      real* x = u + rd.offset;
      const int N = static_cast<int>(rd.N);
      const real c1 = kparam<real>(rd.c1, rd.c1_f), cN = kparam<real>(rd.cN, rd.cN_f);
      const Coef<real> coef{kparam<real>(rd.r, rd.r_f), kparam<real>(one, one_f)};
      real v[E];
      unsigned fixed = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        real y = p < N && index_ok(a.status, rd.offset + p, a.u_len) ? x[p] : static_cast<real>(0);
        if (p == 0) y = c1;
        if (p == N - 1) y = cN;
        v[e] = y;
        if (p == 0 || p == N - 1) fixed |= 1u << e;  // the Dirichlet ends only
      }
      // warps wholly past u_N idle; the others step every position
      const int mode = Win::pos(warp, 0, 0) >= N ? static_cast<int>(kTileIdle) : tile_mode_slot<E>(fixed);
      for (int64_t k0 = 0; k0 < rd.K; k0 += (1 << 30)) {
        const int steps = static_cast<int>(std::min<int64_t>(rd.K - k0, 1 << 30));
        warp_advance_slots<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwarps, blockDim.x, steps);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (p < N && Win::owner(warp, lane, e, nwarps) && index_ok(a.status, rd.offset + p, a.u_len)) x[p] = v[e];
      }
    } else if (kAsync) {
      // One part of a rod run asynchronously: the tile as in the synchronous
      // part below; after each block of T steps the part publishes its first
      // and last T points as strip version j+1 (a ring of R versions per
      // part, release-stored version counter) and starts block j+1 with its
      // neighbours' newest strips not newer than j+1 (at most q-1 blocks old;
      // the recorded ones in a replay), as the blocked asynchronous kernel
      // does for the segments of one rod.
      const BatchRod rd = a.rods[it.rod];
      real* x = u + rd.offset;
      const int64_t N = rd.N;
      const int T = it.T, L = it.L;
      const int64_t a0 = it.a0;
      const bool first = it.part == 0, last = it.part + 1 == it.nparts;
      const int P = nwarps * Win::D + 2 * Win::H;
      const int lo = first ? 0 : (last ? P - L : T);
      const int hi = lo + L;
      const int tile_end = last ? hi : hi + T;
      const real c1 = kparam<real>(rd.c1, rd.c1_f), cN = kparam<real>(rd.cN, rd.cN_f);
      const Coef<real> coef{kparam<real>(rd.r, rd.r_f), kparam<real>(one, one_f)};
      real* strips = static_cast<real*>(a.strips);
      int* myflag = a.flags + it.slot;
      real v[E];
      unsigned fixed = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        const int64_t g = a0 - lo + p;
        real y = static_cast<real>(0);
        if (p < tile_end && g >= 0 && g < N && index_ok(a.status, rd.offset + g, a.u_len)) y = x[g];
        if (g == 0) y = c1;
        if (g == N - 1) y = cN;
        v[e] = y;
        if (p < tile_end && (g == 0 || g == N - 1)) fixed |= 1u << e;
      }
      const int mode = Win::pos(warp, 0, 0) >= tile_end ? static_cast<int>(kTileIdle) : tile_mode<E>(fixed);
      if (tid == 0) sh_part = PartState{lo, hi, T, it.slot, it.part, it.nparts, rd.K, a0, rd.offset};
      // Strip version `ver` of this part; the CTA barrier inside orders every
      // thread's stores before the release of the version counter.
      auto publish = [&](const PartState& ps, int ver) {
        const int64_t sstride = static_cast<int64_t>(a.R) * 2 * a.Tmax;  // values per part
        const int64_t mine0 = ps.slot * sstride + static_cast<int64_t>(ver & (a.R - 1)) * 2 * a.Tmax;
        if (Win::touches(warp, ps.lo, ps.lo + ps.T) || Win::touches(warp, ps.hi - ps.T, ps.hi)) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int p = Win::pos(warp, lane, e);
            if (!Win::owner(warp, lane, e, nwarps)) continue;
            if (p >= ps.lo && p < ps.lo + ps.T && index_ok(a.status, mine0 + (p - ps.lo), a.strips_len))
              st_cg(strips + mine0 + (p - ps.lo), v[e]);
            if (p >= ps.hi - ps.T && p < ps.hi &&
                index_ok(a.status, mine0 + a.Tmax + (p - (ps.hi - ps.T)), a.strips_len))
              st_cg(strips + mine0 + a.Tmax + (p - (ps.hi - ps.T)), v[e]);
          }
        }
        __syncthreads();
        if (tid == 0 && ps.slot != a.stall_slot) st_release_gpu(a.pver + ps.slot, ver);
      };
      __syncthreads();  // every thread has loaded its points; sh_part written
      if (tid == 0) st_release_gpu(myflag, 1);  // loaded: neighbours may now overwrite their own points
      publish(load_part(sh_part), 0);           // version 0: the initial state
      bool ok = true;
      for (int j = 0;; ++j) {
        if (j > 0) {  // block 0 runs on the initial halos (version 0)
          const PartState ps = load_part(sh_part);
          if (tid == 0 || tid == 32 || (blockDim.x <= 32 && tid == 0)) {
            const int64_t toff = a.toff[ps.slot];
            const bool left = tid == 0;
            int ver = j;
            if (left && ps.part > 0) ver = part_strip_version(a, a.pver + ps.slot - 1, j, toff + 2 * j + 0);
            if (!left && ps.part + 1 < ps.nparts) ver = part_strip_version(a, a.pver + ps.slot + 1, j, toff + 2 * j + 1);
            sh_v[left ? 0 : 1] = ver;
            if (blockDim.x <= 32) {  // one-warp CTA: thread 0 takes both sides
              int vr = j;
              if (ps.part + 1 < ps.nparts) vr = part_strip_version(a, a.pver + ps.slot + 1, j, toff + 2 * j + 1);
              sh_v[1] = vr;
            }
          }
          __syncthreads();
          const int vl = sh_v[0], vr = sh_v[1];
          if (vl < 0 || vr < 0) {  // CTA-uniform: every thread reads the same words
            ok = false;
            break;
          }
          const int64_t sstride = static_cast<int64_t>(a.R) * 2 * a.Tmax;
          if (ps.part > 0 && Win::touches(warp, ps.lo - ps.T, ps.lo)) {
            const int64_t left0 = (ps.slot - 1) * sstride + static_cast<int64_t>(vl & (a.R - 1)) * 2 * a.Tmax + a.Tmax;
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int p = Win::pos(warp, lane, e);
              if (p >= ps.lo - ps.T && p < ps.lo && index_ok(a.status, left0 + (p - (ps.lo - ps.T)), a.strips_len))
                v[e] = ld_cg(strips + left0 + (p - (ps.lo - ps.T)));
            }
          }
          if (ps.part + 1 < ps.nparts && Win::touches(warp, ps.hi, ps.hi + ps.T)) {
            const int64_t right0 = (ps.slot + 1) * sstride + static_cast<int64_t>(vr & (a.R - 1)) * 2 * a.Tmax;
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int p = Win::pos(warp, lane, e);
              if (p >= ps.hi && p < ps.hi + ps.T && index_ok(a.status, right0 + (p - ps.hi), a.strips_len))
                v[e] = ld_cg(strips + right0 + (p - ps.hi));
            }
          }
        }
        int tb;
        {
          const PartState ps = load_part(sh_part);
          tb = static_cast<int>(std::min<int64_t>(ps.T, ps.K - static_cast<int64_t>(j) * ps.T));
        }
        warp_advance<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwarps, blockDim.x, tb);
        const PartState ps = load_part(sh_part);
        if (static_cast<int64_t>(j) * ps.T + tb >= ps.K) break;
        // (the barrier inside also keeps sh_v stable until every thread has read it)
        publish(ps, j + 1);
      }
      if (!ok) return;  // CTA-uniform; the status word holds the failure
      const PartState ps = load_part(sh_part);
      int* pflag = a.flags + ps.slot;
      // The neighbours must have loaded their halos before our points change.
      if (tid == 0) {
        bool w = true;
        if (ps.part > 0) w = wait_flag_at_least(pflag - 1, 1, a.status, a.spin_limit_ns);
        if (w && ps.part + 1 < ps.nparts) w = wait_flag_at_least(pflag + 1, 1, a.status, a.spin_limit_ns);
        sh_ok = w;
      }
      __syncthreads();
      if (!sh_ok) return;
      real* px = u + ps.offset;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (p >= ps.lo && p < ps.hi && Win::owner(warp, lane, e, nwarps) &&
            index_ok(a.status, ps.offset + ps.a0 - ps.lo + p, a.u_len))
          px[ps.a0 - ps.lo + p] = v[e];
      }
    } else {
      // One part: position p holds rod point a0 - lo + p, owned points
      // [lo, hi), halos [lo - T, lo) and [hi, hi + T).  As in the synchronous
      // kernel the first part starts at u_1 (lo = 0) and the last part ends at
      // u_N in the CTA's last position, so that both Dirichlet ends sit in
      // slots known at compile time.
      const BatchRod rd = a.rods[it.rod];
      real* x = u + rd.offset;
      const int64_t N = rd.N;
      const int T = it.T, L = it.L;
      const int64_t a0 = it.a0;
      const bool first = it.part == 0, last = it.part + 1 == it.nparts;
      const int P = nwarps * Win::D + 2 * Win::H;
      const int lo = first ? 0 : (last ? P - L : T);
      const int hi = lo + L;
      const int tile_end = last ? hi : hi + T;
      const real c1 = kparam<real>(rd.c1, rd.c1_f), cN = kparam<real>(rd.cN, rd.cN_f);
      const Coef<real> coef{kparam<real>(rd.r, rd.r_f), kparam<real>(one, one_f)};
      int* myflag = a.flags + it.slot;
      real v[E];
      unsigned fixed = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        const int64_t g = a0 - lo + p;
        real y = static_cast<real>(0);
        if (p < tile_end && g >= 0 && g < N && index_ok(a.status, rd.offset + g, a.u_len)) y = x[g];
        if (g == 0) y = c1;
        if (g == N - 1) y = cN;
        v[e] = y;
        if (p < tile_end && (g == 0 || g == N - 1)) fixed |= 1u << e;
      }
      const int mode = Win::pos(warp, 0, 0) >= tile_end ? static_cast<int>(kTileIdle) : tile_mode<E>(fixed);
      if (tid == 0) sh_part = PartState{lo, hi, T, it.slot, it.part, it.nparts, rd.K, a0, rd.offset};
      __syncthreads();
      if (tid == 0) st_release_gpu(myflag, 1);  // loaded: neighbours may now overwrite their own points
      bool ok = true;
      for (int epoch = 0;; ++epoch) {
        int tb;
        {
          const PartState ps = load_part(sh_part);
          tb = static_cast<int>(std::min<int64_t>(ps.T, ps.K - static_cast<int64_t>(epoch) * ps.T));
        }
        warp_advance<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwarps, blockDim.x, tb);
        const PartState ps = load_part(sh_part);
        if (static_cast<int64_t>(epoch) * ps.T + tb >= ps.K) break;
        const int pT = ps.T, plo = ps.lo, phi = ps.hi;
        const size_t estride = static_cast<size_t>(4) * a.Tmax;
        int* pflag = a.flags + ps.slot;
        const int64_t mine0 = ps.slot * static_cast<int64_t>(estride) + (epoch & 1) * 2 * a.Tmax;
        real* mine = edges + mine0;
        if (Win::touches(warp, plo, plo + pT) || Win::touches(warp, phi - pT, phi)) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int p = Win::pos(warp, lane, e);
            if (!Win::owner(warp, lane, e, nwarps)) continue;
            if (p >= plo && p < plo + pT && index_ok(a.status, mine0 + (p - plo), a.edges_len)) st_cg(mine + (p - plo), v[e]);
            if (p >= phi - pT && p < phi && index_ok(a.status, mine0 + a.Tmax + (p - (phi - pT)), a.edges_len))
              st_cg(mine + a.Tmax + (p - (phi - pT)), v[e]);
          }
        }
        __syncthreads();
        if (tid == 0) {
          // A release at GPU scope after the CTA barrier orders every thread's
          // edge stores before the flag (cumulativity); no separate fence.
          if (ps.slot != a.stall_slot) st_release_gpu(pflag, epoch + 2);
          bool w = true;
          if (ps.part > 0) w = wait_flag_at_least(pflag - 1, epoch + 2, a.status, a.spin_limit_ns);
          if (w && ps.part + 1 < ps.nparts) w = wait_flag_at_least(pflag + 1, epoch + 2, a.status, a.spin_limit_ns);
          sh_ok = w;
        }
        __syncthreads();
        if (!sh_ok) {
          ok = false;
          break;
        }
        if (ps.part > 0 && Win::touches(warp, plo - pT, plo)) {
          const int64_t left0 = (ps.slot - 1) * static_cast<int64_t>(estride) + (epoch & 1) * 2 * a.Tmax + a.Tmax;
          const real* left = edges + left0;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int p = Win::pos(warp, lane, e);
            if (p >= plo - pT && p < plo && index_ok(a.status, left0 + (p - (plo - pT)), a.edges_len))
              v[e] = ld_cg(left + (p - (plo - pT)));
          }
        }
        if (ps.part + 1 < ps.nparts && Win::touches(warp, phi, phi + pT)) {
          const int64_t right0 = (ps.slot + 1) * static_cast<int64_t>(estride) + (epoch & 1) * 2 * a.Tmax;
          const real* right = edges + right0;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int p = Win::pos(warp, lane, e);
            if (p >= phi && p < phi + pT && index_ok(a.status, right0 + (p - phi), a.edges_len))
              v[e] = ld_cg(right + (p - phi));
          }
        }
      }
      if (!ok) return;  // CTA-uniform (sh_ok); the status word holds the failure
      const PartState ps = load_part(sh_part);
      int* pflag = a.flags + ps.slot;
      // The neighbours must have loaded their halos before our points change.
      if (tid == 0) {
        bool w = true;
        if (ps.part > 0) w = wait_flag_at_least(pflag - 1, 1, a.status, a.spin_limit_ns);
        if (w && ps.part + 1 < ps.nparts) w = wait_flag_at_least(pflag + 1, 1, a.status, a.spin_limit_ns);
        sh_ok = w;
      }
      __syncthreads();
      if (!sh_ok) return;
      real* px = u + ps.offset;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = Win::pos(warp, lane, e);
        if (p >= ps.lo && p < ps.hi && Win::owner(warp, lane, e, nwarps) &&
            index_ok(a.status, ps.offset + ps.a0 - ps.lo + p, a.u_len))
          px[ps.a0 - ps.lo + p] = v[e];
      }
    }
    __syncthreads();
  }
}

template <typename real, int E>
int launch_batched_t(const BatchRun& a, int threads, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = a.async_mode ? cudaLaunchKernelEx(&cfg, batched_kernel<real, E, true>, a)
                               : cudaLaunchKernelEx(&cfg, batched_kernel<real, E, false>, a);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

template <typename real, int E>
int resident_batched_t(int threads) {
  int per_sm = 0, dev = 0, nsm = 0;
  // the residency of the smaller of the two instances (both must fit the grid)
  int per_sm_async = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<real, E, false>, threads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_async, batched_kernel<real, E, true>, threads, 0) !=
          cudaSuccess)
    return 0;
  per_sm = std::min(per_sm, per_sm_async);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace

}  // namespace heat1d_impl

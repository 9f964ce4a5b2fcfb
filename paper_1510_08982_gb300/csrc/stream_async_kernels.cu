// stream_async_kernels.cu -- the asynchronous run with temporal blocking for
// rods too long to stay on chip: the bounded-delay model of Section 3 (Eq.
// (eqn:async)) applied to blocks of T steps, with the HBM tiles as segments.
//
// The rod is cut into tiles of W points (the last one shorter); tile j is the
// segment [jW, min((j+1)W, N)).  In block b a tile advances T steps on its own
// points at step bT and two halo strips: its left neighbour's last T points
// and its right neighbour's first T points at step (b - d)T, d < q -- the
// newest versions published, waiting only while one is more than q-1 blocks
// old.  Its own points after the block are written back in place (no other
// tile reads them) and its first and last Th >= T points are published as
// strip version b+1 into a ring of R versions per tile, followed by a release
// store of the tile's version counter.  The delay of every strip read is
// recorded, and a replay waits for exactly version b - d.  No grid barrier and
// no pass ordering beyond the delay window: a tile runs ahead of a slow
// neighbour by up to q-1 blocks.
//
// The pipeline is the streamed synchronous kernel's: a loader thread picks
// the strip versions, then copies the tile's own points and the two strips
// into a shared-memory stage by bulk copies (1D TMA) completing on the stage's
// mbarrier; the compute warps advance the stage in registers and store it;
// a releaser thread publishes the version.  The last tile (which may be
// shorter than W) is loaded with plain loads.  Every wait is bounded.
//
// Ring safety: a tile starts block b only after both neighbours published
// version b-q+1, so neighbours drift at most q-1 blocks apart; a reader in
// block b needs versions >= b-q+1 while a writer has published at most b+q,
// whose slot held version b+q-R < b-q+1 whenever R >= 2q.
#include <algorithm>

#include "bulk.cuh"
#include "checked.cuh"
#include "common.cuh"
#include "impl.h"

namespace heat1d_impl {
using namespace heat1d_dev;

namespace {

// Chooses (free run) or looks up (replay) the neighbour version that block b
// reads and waits for it to be published.  One thread.  Returns the version,
// or -1 after raising a failure.
__device__ int tile_strip_version(const StreamAsyncRun& a, const int* nb_ver, int b, size_t tidx) {
  int need;
  if (a.trace_in) {
    const int d = index_ok(a.status, static_cast<int64_t>(tidx), a.trace_len) ? a.trace_in[tidx] : 0;
    if (d >= a.q) {
      raise_status(a.status, HEAT1D_ERR_TRACE);
      return -1;
    }
    need = b - min(d, b);
  } else {
    need = max(b - a.q + 1, 0);
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
      __nanosleep(64);
    }
  }
  const int v = a.trace_in ? need : min(V, b);
  if (a.trace_out && index_ok(a.status, static_cast<int64_t>(tidx), a.trace_len))
    a.trace_out[tidx] = static_cast<uint8_t>(b - v);
  return v;
}

// Waits until a tile's version counter reaches `want`.
__device__ bool wait_version(const int* ver, int want, int* status, int64_t limit_ns) {
  if (ld_acquire_gpu(ver) >= want) return true;
  const uint64_t t0 = global_timer_ns();
  unsigned spins = 0;
  while (ld_acquire_gpu(ver) < want) {
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

// Version 0 of every tile's strips is the initial state.
template <typename real>
__global__ void stream_async_setup_kernel(StreamAsyncRun a) {
  const real* u = static_cast<const real*>(a.u);
  real* strips = static_cast<real*>(a.strips);
  const int Th = a.Th;
  for (int64_t j = blockIdx.x; j < a.ntiles; j += gridDim.x) {
    const int64_t lo = j * a.W;
    const int64_t L = std::min<int64_t>(a.W, a.N - lo);
    const int64_t s00 = j * a.R * 2 * Th;
    real* s0 = strips + s00;  // version 0 sits in slot 0
    for (int i = threadIdx.x; i < Th; i += blockDim.x) {
      const int64_t gf = lo + i, gl = lo + L - Th + i;
      if (index_ok(a.status, s00 + i, a.strips_len))
        s0[i] = gf < a.N && index_ok(a.status, gf, a.N) ? u[gf] : static_cast<real>(0);
      if (index_ok(a.status, s00 + Th + i, a.strips_len))
        s0[Th + i] = gl >= 0 && index_ok(a.status, gl, a.N) ? u[gl] : static_cast<real>(0);
    }
    if (threadIdx.x == 0) a.ver[j] = 0;
  }
}

template <typename real, int E>
__global__ void __launch_bounds__(kStreamMaxThreads + 64, 1) stream_async_kernel(StreamAsyncRun a) {
  using V = typename Vec16<real>::type;
  using Win = Window<E, stream_window_halo(sizeof(real), E)>;
  constexpr int VN = Vec16<real>::n;
  static_assert(E % VN == 0, "E must be a multiple of the 16-byte vector width");
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ WindowShared<real, Win::H> sh;
  __shared__ __align__(8) uint64_t full[kStages], stored[kStages], freed[kStages];
  __shared__ int stage_plain[kStages], stage_vl[kStages], stage_vr[kStages];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwc = (blockDim.x >> 5) - 2;  // compute warps; then the loader and the releaser warp
  const unsigned nthreads_c = static_cast<unsigned>(nwc) * 32u;
  const int64_t N = a.N;
  const int Th = a.Th, W = a.W, Wt = a.W + 2 * a.Th;
  const int R = a.R;
  real* stage0 = reinterpret_cast<real*>(dyn);
  real* u = static_cast<real*>(a.u);
  real* strips = static_cast<real*>(a.strips);
  const int nblocks = static_cast<int>((a.K + a.T - 1) / a.T);
  const int64_t nbnd = a.ntiles - 1;  // boundaries per block in the trace
  const int64_t my_tiles = a.ntiles > blockIdx.x ? (a.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // Items in order: every block, this CTA's tiles blockIdx.x, blockIdx.x + G, ...
  const int64_t items = my_tiles * nblocks;

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
    int b = 0, st = 0;
    unsigned round = 0;
    int64_t j = blockIdx.x;
    for (int64_t i = 0; i < items; ++i) {
      if (round > 0 && !mbar_wait(&freed[st], (round - 1) & 1u, a.status, a.spin_limit_ns, true)) break;
      // The tile's own points of block b were stored by this CTA's compute
      // warps in block b-1; with at least kStages tiles per CTA the wait on
      // "freed" above already covers that item.
      if (b > 0 && my_tiles < kStages && !wait_version(a.ver + j, b, a.status, a.spin_limit_ns)) break;
      int vl = -1, vr = -1;
      if (j > 0) {
        vl = tile_strip_version(a, a.ver + (j - 1), b, (static_cast<size_t>(b) * nbnd + (j - 1)) * 2 + 1);
        if (vl < 0) break;
      }
      if (j + 1 < a.ntiles) {
        vr = tile_strip_version(a, a.ver + (j + 1), b, (static_cast<size_t>(b) * nbnd + j) * 2 + 0);
        if (vr < 0) break;
      }
      const bool plain = j + 1 == a.ntiles;  // the last tile may be shorter than W
      stage_plain[st] = plain;
      stage_vl[st] = vl;
      stage_vr[st] = vr;
      if (plain) {
        mbar_arrive(&full[st]);  // release: the waits and the words above come first
      } else {
        // The strips and own points were stored through the generic proxy;
        // the copies read through the async proxy, and the stage's previous
        // contents were read through the generic proxy.
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        real* stg = stage0 + static_cast<size_t>(st) * Wt;
        const unsigned hb = static_cast<unsigned>(Th) * sizeof(real), ob = static_cast<unsigned>(W) * sizeof(real);
        const unsigned bytes = ob + (vl >= 0 ? hb : 0u) + hb;
        mbar_arrive_expect_tx(&full[st], bytes);
        // (checked build: a copy whose range leaves its buffer is skipped; its
        // stage then never fills and the compute warps' bounded wait ends the run)
        const int64_t ls0 = ((static_cast<int64_t>(j - 1) * R + (vl & (R - 1))) * 2 + 1) * Th;
        const int64_t rs0 = (static_cast<int64_t>(j + 1) * R + (vr & (R - 1))) * 2 * Th;
        if (index_ok(a.status, j * W, N) && index_ok(a.status, j * W + W - 1, N))
          bulk_copy_to_shared(stg + Th, u + j * W, ob, &full[st]);
        if (vl >= 0 && index_ok(a.status, ls0, a.strips_len) && index_ok(a.status, ls0 + Th - 1, a.strips_len))
          bulk_copy_to_shared(stg, strips + ls0, hb, &full[st]);  // the left neighbour's last Th points
        if (index_ok(a.status, rs0, a.strips_len) && index_ok(a.status, rs0 + Th - 1, a.strips_len))
          bulk_copy_to_shared(stg + Th + W, strips + rs0, hb, &full[st]);  // the right neighbour's first Th points
      }
      issued = i + 1;
      j += gridDim.x;
      if (j >= a.ntiles) {
        j = blockIdx.x;
        ++b;
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
    int b = 0, st = 0;
    unsigned round = 0;
    int64_t j = blockIdx.x;
    for (int64_t i = 0; i < items; ++i) {
      if (!mbar_wait(&stored[st], round & 1u, a.status, a.spin_limit_ns, true)) break;
      // Release at GPU scope after the compute warps' arrivals: their stores
      // of the tile and of its strips come first (cumulativity).
      if (j != a.stall_tile) st_release_gpu(a.ver + j, b + 1);
      mbar_arrive(&freed[st]);
      j += gridDim.x;
      if (j >= a.ntiles) {
        j = blockIdx.x;
        ++b;
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
  int b = 0, st = 0;
  unsigned round = 0;
  int64_t j = blockIdx.x;
  for (int64_t i = 0; i < items; ++i) {
    const int tb = static_cast<int>(std::min<int64_t>(a.T, a.K - static_cast<int64_t>(b) * a.T));
    bool failed = !mbar_wait(&full[st], round & 1u, a.status, a.spin_limit_ns, true);
    const int64_t lo = j * W;
    const int L = static_cast<int>(std::min<int64_t>(W, N - lo));
    const int64_t g0 = lo - Th;  // stage position p holds point g0 + p
    const int64_t gt = g0 + p0;
    // No Dirichlet end anywhere in the stage: every position steps freely.
    const bool inner = g0 > 0 && g0 + Wt < N;
    real v[E];
    if (!failed && !stage_plain[st]) {
      const real* sp = stage0 + static_cast<size_t>(st) * Wt + p0;
#pragma unroll
      for (int qq = 0; qq < E / VN; ++qq) {
        const V x = reinterpret_cast<const V*>(sp)[qq];
        const real* xs = reinterpret_cast<const real*>(&x);
#pragma unroll
        for (int t = 0; t < VN; ++t) v[qq * VN + t] = xs[t];
      }
    } else {
      const int vl = stage_vl[st], vr = stage_vr[st];
      const int64_t sl0 = ((static_cast<int64_t>(j - 1) * R + (vl & (R - 1))) * 2 + 1) * Th;
      const int64_t sr0 = (static_cast<int64_t>(j + 1) * R + (vr & (R - 1))) * 2 * Th;
      const real* sl = vl >= 0 ? strips + sl0 : nullptr;
      const real* sr = vr >= 0 ? strips + sr0 : nullptr;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = p0 + e;
        const int64_t g = gt + e;
        real x = static_cast<real>(0);
        if (!failed) {
          if (p < Th) {
            if (sl && index_ok(a.status, sl0 + p, a.strips_len)) x = ld_cg(sl + p);
          } else if (p < Th + L) {
            if (index_ok(a.status, g, N)) x = ld_cg(u + g);
          } else if (p < Th + W + Th && p >= Th + W) {
            if (sr && index_ok(a.status, sr0 + (p - Th - W), a.strips_len)) x = ld_cg(sr + (p - Th - W));
          }
        }
        v[e] = x;
      }
    }
    // A failed wait ends the run for every compute warp (see the streamed
    // synchronous kernel: passes longer than H steps meet refresh barriers).
    // The last tile reads its own points straight from the state it updates
    // in place, and adjacent warps both load the points their windows share:
    // every warp must have loaded before any warp stores, so that tile always
    // meets this barrier (the value is the same for the whole CTA).
    if (a.T > Win::H || stage_plain[st]) {
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
        if (g == 0 || g == N - 1) fixed |= 1u << e;
      }
      const int mode = tile_mode<E>(fixed);
      warp_advance<real, E, Win::H>(mode, v, fixed, coef, sh, parity, warp, lane, nwc, nthreads_c, tb, false);
    }
    // Own points back in place, and strip version b+1: the first Th and the
    // last Th own points.
    if (owns_all && p0 >= Th && p0 + E <= Th + L && index_ok(a.status, gt, N) && index_ok(a.status, gt + E - 1, N)) {
#pragma unroll
      for (int qq = 0; qq < E / VN; ++qq) {
        V x;
        real* xs = reinterpret_cast<real*>(&x);
#pragma unroll
        for (int t = 0; t < VN; ++t) xs[t] = v[qq * VN + t];
        __stcg(reinterpret_cast<V*>(u + gt) + qq, x);
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = p0 + e;
        if (p >= Th && p < Th + L && Win::owner(warp, lane, e, nwc) && index_ok(a.status, gt + e, N))
          __stcg(u + gt + e, v[e]);
      }
    }
    if (b + 1 < nblocks) {
      const int64_t sv0 = (static_cast<int64_t>(j) * R + ((b + 1) & (R - 1))) * 2 * Th;
      real* sv = strips + sv0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int p = p0 + e;
        if (!Win::owner(warp, lane, e, nwc)) continue;
        if (p >= Th && p < 2 * Th && index_ok(a.status, sv0 + (p - Th), a.strips_len)) st_cg(sv + (p - Th), v[e]);
        if (p >= L && p < L + Th && index_ok(a.status, sv0 + Th + (p - L), a.strips_len)) st_cg(sv + Th + (p - L), v[e]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&stored[st]);  // release: this warp's stores come first
    j += gridDim.x;
    if (j >= a.ntiles) {
      j = blockIdx.x;
      ++b;
    }
    if (++st == kStages) {
      st = 0;
      ++round;
    }
  }
}

template <typename real>
size_t async_smem_bytes(int Wt) {
  return static_cast<size_t>(kStages) * Wt * sizeof(real);
}

template <typename real, int E>
int launch_t(const StreamAsyncRun& a, int threads, int grid, cudaStream_t st) {
  StreamAsyncRun args = a;
  set_run_params(args);
  void* params[] = {&args};
  const size_t smem = async_smem_bytes<real>(a.W + 2 * a.Th);
  if (cudaFuncSetAttribute(stream_async_kernel<real, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return HEAT1D_ERR_CUDA;
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(stream_async_kernel<real, E>), dim3(grid),
                                              dim3(threads + 64), params, smem, st);
  if (e == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    return HEAT1D_ERR_NOT_RESIDENT;
  }
  return e == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

template <typename real, int E>
int resident_t(int threads, int Wt) {
  int per_sm = 0, dev = 0, nsm = 0;
  const size_t smem = async_smem_bytes<real>(Wt);
  if (cudaFuncSetAttribute(stream_async_kernel<real, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_async_kernel<real, E>, threads + 64, smem) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * nsm;
}

}  // namespace

int launch_stream_async_setup(const StreamAsyncRun& a, int dtype, cudaStream_t st) {
  const int grid = static_cast<int>(std::min<int64_t>(a.ntiles, 4096));
  if (dtype == HEAT1D_F64)
    stream_async_setup_kernel<double><<<grid, 128, 0, st>>>(a);
  else
    stream_async_setup_kernel<float><<<grid, 128, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? HEAT1D_OK : HEAT1D_ERR_CUDA;
}

int launch_stream_async(const StreamAsyncRun& a, int dtype, int E, int threads, int grid, cudaStream_t st) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 4: return f64 ? launch_t<double, 4>(a, threads, grid, st) : launch_t<float, 4>(a, threads, grid, st);
    case 8: return f64 ? launch_t<double, 8>(a, threads, grid, st) : launch_t<float, 8>(a, threads, grid, st);
    case 16: return f64 ? launch_t<double, 16>(a, threads, grid, st) : launch_t<float, 16>(a, threads, grid, st);
    default: return HEAT1D_ERR_INVAL;
  }
}

int max_resident_stream_async(int dtype, int E, int threads, int Wt) {
  const bool f64 = dtype == HEAT1D_F64;
  switch (E) {
    case 4: return f64 ? resident_t<double, 4>(threads, Wt) : resident_t<float, 4>(threads, Wt);
    case 8: return f64 ? resident_t<double, 8>(threads, Wt) : resident_t<float, 8>(threads, Wt);
    case 16: return f64 ? resident_t<double, 16>(threads, Wt) : resident_t<float, 16>(threads, Wt);
    default: return 0;
  }
}

}  // namespace heat1d_impl

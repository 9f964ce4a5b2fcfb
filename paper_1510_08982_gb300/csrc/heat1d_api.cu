// heat1d_api.cu -- the C ABI of libheat1d (declared in include/heat1d.h).
//
// Argument checks, the segment split, scratch-buffer ownership and the choice
// of launch shape live here; every step of the computation runs in the
// kernels of sync_kernels.cu and async_kernels.cu.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "checked.cuh"
#include "heat1d.h"
#include "impl.h"

using heat1d_impl::SegmentRun;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return HEAT1D_ERR_CUDA;
}

#define HEAT1D_CUDA(call)                                \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Sets the two Dirichlet ends of a device state (Section 2: u_1 = c1, u_N = cN).
template <typename real>
__global__ void set_ends_kernel(real* u, int64_t N, double c1, double cN) {
  if (threadIdx.x == 0) u[0] = static_cast<real>(c1);
  if (threadIdx.x == 1) u[N - 1] = static_cast<real>(cN);
}


// History of a state that does not continue an asynchronous run: every
// entry is the segment's current edge value (a run started from it reads no
// step before it).
template <typename real>
__global__ void edges_history_kernel(const real* u, const int64_t* off, int S, int q, real* hist) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const real first = u[off[s]], last = u[off[s + 1] - 1];
    for (int j = 0; j < q; ++j) {
      hist[(static_cast<size_t>(s) * 2 + 0) * q + j] = first;
      hist[(static_cast<size_t>(s) * 2 + 1) * q + j] = last;
    }
  }
}

// Checked build only: one load and one store at index n (one past the end
// of buf); the checks skip both and record HEAT1D_ERR_BOUNDS.  The index is
// computed on the device so that no compiler can drop the checks.
__global__ void checked_selftest_kernel(double* buf, int n, int* status) {
  if constexpr (heat1d_dev::kChecked) {
    if (threadIdx.x != 0) return;
    const int i = n + static_cast<int>(blockIdx.x);  // = n
    double x = 0.0;
    if (heat1d_dev::index_ok(status, i, n)) x = buf[i];
    if (heat1d_dev::index_ok(status, i, n)) buf[i] = x + 1.0;
  }
}

constexpr int64_t kStateMagic = 0x3144485453453148LL;  // "H1ESTHD1"

}  // namespace

void heat1d_impl::set_last_error(const std::string& msg) { g_last_error = msg; }

struct heat1d {
  int64_t N = 0;
  double r = 0, c1 = 0, cN = 0;
  int dtype = HEAT1D_F64;
  size_t esize = 8;
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  heat1d_opts opts{};

  // resolved configuration
  int S = 1, q = 3, R = 8, T = 1;
  // streamed synchronous run: steps per pass, halo, tile shape
  int Ts = 8, Th = 8, sE = 8, sthreads = 256, W = 0;
  int64_t ntiles = 0;
  std::vector<int64_t> off;
  int64_t Lmin = 0, Lmax = 0;

  // device memory (owned)
  void* u[2] = {nullptr, nullptr};
  int cur = 0;
  int64_t* d_off = nullptr;
  void* edges = nullptr;
  void* rings = nullptr;
  int* prog = nullptr;
  int* done = nullptr;  // streamed run: passes completed per tile
  void* ctl = nullptr;  // [0]: grid barrier counter, [32]: status word (separate lines)
  uint8_t* d_trace = nullptr;
  size_t d_trace_bytes = 0;
  void* snap = nullptr;  // caller's snapshot buffer (device) or null
  int64_t snap_every = 0, snap_rows = 0;
  void* strips = nullptr;  // blocked asynchronous run: [S][R][2T] strips, allocated on first use
  size_t strips_bytes = 0;
  // Checkpoint/resume of the asynchronous run: the current state is global
  // step async_step of an asynchronous run whose segments' edge values at
  // its last q steps are in hist[hist_cur] ([S][2][q]); hist_cur < 0: no
  // such history (the next asynchronous run starts at step 0).
  int64_t async_step = 0;
  void* hist[2] = {nullptr, nullptr};
  size_t hist_bytes = 0;
  int hist_cur = -1;

  unsigned* barrier() { return static_cast<unsigned*>(ctl); }
  int* status() { return static_cast<int*>(ctl) + 32; }
};

namespace {

// The state no longer continues an asynchronous run (a new u, another kind
// of run, new options).
void reset_history(heat1d* h) {
  h->async_step = 0;
  h->hist_cur = -1;
}

void free_scratch(heat1d* h) {
  cudaFree(h->hist[0]);
  cudaFree(h->hist[1]);
  h->hist[0] = h->hist[1] = nullptr;
  h->hist_bytes = 0;
  reset_history(h);
  cudaFree(h->d_off);
  cudaFree(h->edges);
  cudaFree(h->rings);
  cudaFree(h->prog);
  cudaFree(h->done);
  cudaFree(h->strips);
  h->strips = nullptr;
  h->strips_bytes = 0;
  h->d_off = nullptr;
  h->edges = nullptr;
  h->rings = nullptr;
  h->prog = nullptr;
  h->done = nullptr;
}

// Resolves the options against N and (re)allocates the scratch buffers.
int configure(heat1d* h, const heat1d_opts& o) {
  if (o.segments < 0 || o.q < 0 || o.q > 255 || o.halo_steps < 0 || o.block_threads < 0 ||
      o.elems_per_thread < 0 || o.spin_limit_ns < 0)
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: negative or out-of-range option");
  if (o.elems_per_thread && o.elems_per_thread != 2 && o.elems_per_thread != 4 && o.elems_per_thread != 8 &&
      o.elems_per_thread != 16 && !(o.elems_per_thread == 32 && h->esize == 4))
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: elems_per_thread must be 2, 4, 8 or 16 (or 32 in F32)");
  if (o.block_threads % 32 != 0 || o.block_threads > 1024)
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: block_threads must be a multiple of 32, at most 1024");
  int64_t S = o.segments ? o.segments : h->nsm;
  S = std::min<int64_t>(S, h->N);
  if (S < 1 || S > INT_MAX) return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: bad segment count");

  std::vector<int64_t> off(S + 1);
  const int64_t base = h->N / S, extra = h->N % S;
  int64_t pos = 0;
  for (int64_t s = 0; s < S; ++s) {
    off[s] = pos;
    pos += base + (s < extra ? 1 : 0);
  }
  off[S] = pos;
  const int64_t Lmax = base + (extra ? 1 : 0), Lmin = base;

  const int q = o.q ? o.q : 3;
  int R = 1;
  while (R < 2 * q) R <<= 1;
  if (R > heat1d_impl::kMaxRing) return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: q too large");
  // On-chip synchronous runs take halos from the neighbouring segment only,
  // so their T is at most the shortest segment (clamped unless on-chip mode
  // was asked for explicitly).
  // Default depth (measured best on GB300): FP32 512 steps on segments of
  // 6144 points or more, 256 from 4096, else 128 -- a step costs little and
  // an exchange (about 5 us a block on the 2^20-point rod) weighs more than
  // the halo's redundant points (on that rod: 6.54e12 updates/s at T = 128,
  // 7.09e12 at 256, 7.33e12 at 512); FP64 64 steps on segments of 4096
  // points or more and 32 on shorter ones, where the redundant arithmetic
  // weighs more (1.80e11 at 32, 1.815e11 at 64, 1.76e11 at 128).
  int T = o.halo_steps ? o.halo_steps
                       : (h->esize == 4 ? (Lmin >= 6144 ? 512 : (Lmin >= 4096 ? 256 : 128))
                                        : (Lmin >= 4096 ? 64 : 32));
  if (T > Lmin) {
    if (o.halo_steps && o.sync_mode == 1)
      return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: halo_steps exceeds the shortest segment");
    T = static_cast<int>(Lmin);
  }
  if (T < 1) T = 1;
  if (o.sync_mode < 0 || o.sync_mode > 2) return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: sync_mode must be 0, 1 or 2");
  if (o.boundary < 0 || o.boundary > 1) return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: boundary must be 0 or 1");
  if (o.boundary == 1 && o.sync_mode == 2)
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: periodic runs are on-chip only (sync_mode 0 or 1)");
  if (o.cluster != 0 && o.cluster != 1 && o.cluster != 2 && o.cluster != 4 && o.cluster != 8)
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: cluster must be 0, 1, 2, 4 or 8");
  if (o.cluster > 1 && S % o.cluster != 0)
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: cluster must divide the number of segments");

  // Streamed shape: 16-byte vectors, so E and the halo are multiples of
  // 16 / sizeof(real) points and every tile starts on a 16-byte boundary.
  const int vn = static_cast<int>(16 / h->esize);
  const int Ts = o.halo_steps ? o.halo_steps : (h->esize == 4 ? 128 : 32);
  const int Th = (Ts + vn - 1) / vn * vn;
  const int sE = o.elems_per_thread ? o.elems_per_thread : (h->esize == 8 ? 8 : 16);
  const int sthreads = o.block_threads ? o.block_threads : 256;
  if (sE % vn != 0 && o.sync_mode == 2)
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: streamed runs need elems_per_thread a multiple of 16 bytes");
  const int64_t W =
      heat1d_impl::window_width(sthreads / 32, sE, heat1d_impl::stream_window_halo(static_cast<int>(h->esize), sE)) - 2 * Th;
  // (the streamed kernel adds one producer warp to the compute threads)
  if (o.sync_mode == 2 && (W < vn || sthreads > heat1d_impl::kStreamMaxThreads))
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_opts: streamed tile too small for halo_steps, or too many threads");
  const int64_t ntiles = W >= vn ? (h->N + W - 1) / W : 0;

  free_scratch(h);
  h->Ts = Ts;
  h->Th = Th;
  h->sE = sE;
  h->sthreads = sthreads;
  h->W = static_cast<int>(W);
  h->ntiles = ntiles;
  h->S = static_cast<int>(S);
  h->q = q;
  h->R = R;
  h->T = T;
  h->off = off;
  h->Lmin = Lmin;
  h->Lmax = Lmax;
  h->opts = o;
  if (h->opts.spin_limit_ns == 0) h->opts.spin_limit_ns = 2000000000LL;
  HEAT1D_CUDA(cudaMalloc(&h->d_off, sizeof(int64_t) * (S + 1)));
  HEAT1D_CUDA(cudaMemcpy(h->d_off, off.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice));
  HEAT1D_CUDA(cudaMalloc(&h->edges, h->esize * 2 * S * 2 * T));
  // tagged slots: one 64-bit word per 32 bits of a value
  HEAT1D_CUDA(cudaMalloc(&h->rings, 2 * h->esize * S * 2 * R));
  HEAT1D_CUDA(cudaMalloc(&h->prog, sizeof(int) * S * heat1d_impl::kProgStride));
  if (ntiles > 0) HEAT1D_CUDA(cudaMalloc(&h->done, sizeof(int) * ntiles));
  return HEAT1D_OK;
}

// The streamed synchronous run (temporal blocking through HBM).
int run_streamed(heat1d* h, int64_t K) {
  if (h->ntiles <= 0 || (h->sE != 4 && h->sE != 8 && h->sE != 16) ||
      h->sthreads > heat1d_impl::kStreamMaxThreads)
    return fail(HEAT1D_ERR_INVAL,
                "streamed run: invalid tile shape (elems_per_thread must be 4, 8 or 16; block_threads at most 512)");
  heat1d_impl::StreamRun a{};
  a.N = h->N;
  a.K = K;
  a.T = h->Ts;
  a.Th = h->Th;
  a.W = h->W;
  a.ntiles = h->ntiles;
  a.u_a = h->u[h->cur];
  a.u_b = h->u[1 - h->cur];
  a.r = h->r;
  a.c1 = h->c1;
  a.cN = h->cN;
  a.done = h->done;
  a.status = h->status();
  a.spin_limit_ns = h->opts.spin_limit_ns;
  a.stall_tile = h->opts.stall_segment;
  // Pipelined kernel: tile loads by bulk copies from one extra producer warp.
  const int resident = heat1d_impl::max_resident_stream_tma(h->dtype, h->sE, h->sthreads, h->W + 2 * h->Th);
  if (resident <= 0) return fail(HEAT1D_ERR_NOT_RESIDENT, "streamed run: kernel cannot be resident");
  const int grid = static_cast<int>(std::min<int64_t>(h->ntiles, resident));
  HEAT1D_CUDA(cudaMemsetAsync(h->done, 0, sizeof(int) * h->ntiles, h->stream));
  int rc = heat1d_impl::launch_stream_tma(a, h->dtype, h->sE, h->sthreads, grid, h->stream);
  if (rc == HEAT1D_ERR_NOT_RESIDENT) return fail(rc, "streamed run: grid cannot be resident");
  if (rc) return cuda_fail(cudaGetLastError(), "launch_stream_tma");
  const int64_t npass = (K + h->Ts - 1) / h->Ts;
  if (npass & 1) h->cur = 1 - h->cur;
  return HEAT1D_OK;
}

// Launch shape for a tile of `slots` positions: the fewest points per thread E
// whose warp count (overlapping warp windows of 32E points, see common.cuh)
// fits the kernel's CTA limit minus `reserved` threads (the asynchronous
// kernel's communication warp), unless E or the thread count is forced.
// Returns false (setting nothing) when no shape fits.
bool try_shape(const heat1d* h, int64_t slots, int reserved, bool async_kernel, int* E, int* threads) {
  const int forced_E = h->opts.elems_per_thread;
  // FP32 tries 16 points per thread first when the tile still spreads over
  // at least 8 warps: per update it then issues half the shuffles and halo
  // refreshes of E = 8, which on GB300 ran 1.2-1.4x faster.
  const bool prefer16 = h->esize == 4 && slots >= 8 * 32 * 16;
  const int Es[5] = {2, 4, 8, 16, 32};
  const int Es16[5] = {16, 2, 4, 8, 32};
  // 32 points per thread: FP32 synchronous-family kernels only
  const int ncand = (h->esize == 4 && !async_kernel) ? 5 : 4;
  for (int i = 0; i < ncand; ++i) {
    const int e = prefer16 ? Es16[i] : Es[i];
    if (forced_E && e != forced_E) continue;
    const int64_t limit = (async_kernel ? heat1d_impl::max_async_threads(static_cast<int>(h->esize), e)
                                        : heat1d_impl::max_tile_threads(static_cast<int>(h->esize), e)) - reserved;
    const int es = static_cast<int>(h->esize);
    const int H = async_kernel ? heat1d_impl::async_window_halo(es, e) : heat1d_impl::sync_window_halo(es, e);
    int64_t t = 32 * heat1d_impl::window_warps(slots, e, H);
    if (h->opts.block_threads) {
      if (h->opts.block_threads < t) continue;
      t = h->opts.block_threads;
    }
    if (t <= limit) {
      *E = e;
      *threads = static_cast<int>(t);
      return true;
    }
  }
  return false;
}

int pick_shape(const heat1d* h, int64_t slots, int reserved, bool async_kernel, int* E, int* threads) {
  if (try_shape(h, slots, reserved, async_kernel, E, threads)) return HEAT1D_OK;
  return fail(HEAT1D_ERR_INVAL,
              "segments too long for the on-chip kernels (" + std::to_string(slots) +
                  " points per CTA); use more segments");
}

// Whether the blocked asynchronous run streams through HBM (tiles as
// segments): asked for with sync_mode 2, or chosen when a segment does not
// fit one CTA (sync_mode 0) on a rod with Dirichlet ends.
bool blocked_streamed(const heat1d* h) {
  if (h->opts.sync_mode == 2) return true;
  if (h->opts.sync_mode == 1 || h->opts.boundary == 1) return false;
  int E = 0, threads = 0;
  return !try_shape(h, h->Lmax + 2 * h->T, 0, false, &E, &threads);
}

SegmentRun base_run(heat1d* h, int64_t K) {
  SegmentRun a{};
  a.N = h->N;
  a.K = K;
  a.S = h->S;
  a.seg_off = h->d_off;
  a.u_in = h->u[h->cur];
  a.u_out = h->u[1 - h->cur];
  a.r = h->r;
  a.c1 = h->c1;
  a.cN = h->cN;
  a.status = h->status();
  a.spin_limit_ns = h->opts.spin_limit_ns;
  a.T = h->T;
  a.edges = h->edges;
  a.barrier = h->barrier();
  a.q = h->q;
  a.R = h->R;
  a.prog = h->prog;
  a.rings = h->rings;
  a.stall_segment = h->opts.stall_segment;
  a.periodic = h->opts.boundary == 1;
  if (h->snap && h->snap_every > 0 && K / h->snap_every + 1 <= h->snap_rows) {
    a.snap = h->snap;
    a.snap_every = h->snap_every;
    a.snap_len = h->snap_rows * h->N;
  }
  a.edges_len = 2 * h->S * 2 * static_cast<int64_t>(h->T);
  a.ring_len = h->S * 2 * static_cast<int64_t>(h->R) * static_cast<int64_t>(h->esize / 4);  // tagged slot words
  a.hist_len = h->S * 2 * static_cast<int64_t>(h->q);
  return a;
}

int ensure_trace_staging(heat1d* h, size_t bytes) {
  if (bytes <= h->d_trace_bytes) return HEAT1D_OK;
  cudaFree(h->d_trace);
  h->d_trace = nullptr;
  h->d_trace_bytes = 0;
  cudaError_t e = cudaMalloc(&h->d_trace, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(trace staging)");
  h->d_trace_bytes = bytes;
  return HEAT1D_OK;
}

// Device addresses of a run's trace buffers (tbytes bytes each; none when
// tbytes is 0, i.e. one segment): a host output trace is written to the
// staging buffer and copied back after the run, a host input trace is copied
// into it before; only one of the two may be on the host.
int stage_traces(heat1d* h, size_t tbytes, uint8_t* trace_out, int out_on_device, const uint8_t* trace_in,
                 int in_on_device, uint8_t** out_dev, const uint8_t** in_dev) {
  int rc;
  *out_dev = nullptr;
  *in_dev = nullptr;
  if (trace_out && tbytes) {
    if (out_on_device) {
      *out_dev = trace_out;
    } else {
      if ((rc = ensure_trace_staging(h, tbytes))) return rc;
      *out_dev = h->d_trace;
    }
  }
  if (trace_in && tbytes) {
    if (in_on_device) {
      *in_dev = trace_in;
    } else {
      if (*out_dev && *out_dev == h->d_trace) return fail(HEAT1D_ERR_INVAL, "host trace in and out at once");
      if ((rc = ensure_trace_staging(h, tbytes))) return rc;
      HEAT1D_CUDA(cudaMemcpyAsync(h->d_trace, trace_in, tbytes, cudaMemcpyHostToDevice, h->stream));
      *in_dev = h->d_trace;
    }
  }
  return HEAT1D_OK;
}

int run_async_common(heat1d* h, int64_t K, uint8_t* trace_out, int out_on_device, const uint8_t* trace_in,
                     int in_on_device) {
  if (K < 0 || K >= INT_MAX) return fail(HEAT1D_ERR_INVAL, "K out of range");
  if (K == 0) return HEAT1D_OK;
  int E = 0, threads = 0;
  int rc = pick_shape(h, h->Lmax + 2, 32 * heat1d_impl::kCommWarps, true, &E, &threads);
  if (rc) return rc;
  if (h->snap && K / h->snap_every + 1 > h->snap_rows)
    return fail(HEAT1D_ERR_INVAL, "snapshot buffer holds fewer rows than K/every + 1");
  const bool periodic = h->opts.boundary == 1;
  if (periodic && h->S < 2) return fail(HEAT1D_ERR_INVAL, "periodic asynchronous runs need at least 2 segments");
  const size_t tbytes = static_cast<size_t>(K) * (periodic ? h->S : h->S - 1) * 2;
  SegmentRun a = base_run(h, K);
  uint8_t* out_dev = nullptr;
  const uint8_t* in_dev = nullptr;
  if ((rc = stage_traces(h, tbytes, trace_out, out_on_device, trace_in, in_on_device, &out_dev, &in_dev))) return rc;
  a.trace_out = out_dev;
  a.trace_in = in_dev;
  a.trace_len = static_cast<int64_t>(tbytes);
  const size_t hbytes = h->esize * static_cast<size_t>(h->S) * 2 * h->q;
  if (hbytes > h->hist_bytes) {
    cudaFree(h->hist[0]);
    cudaFree(h->hist[1]);
    h->hist[0] = h->hist[1] = nullptr;
    h->hist_bytes = 0;
    reset_history(h);
    HEAT1D_CUDA(cudaMalloc(&h->hist[0], hbytes));
    HEAT1D_CUDA(cudaMalloc(&h->hist[1], hbytes));
    h->hist_bytes = hbytes;
  }
  const int hout = h->hist_cur >= 0 ? 1 - h->hist_cur : 0;
  a.k0 = h->hist_cur >= 0 ? h->async_step : 0;
  a.hist_in = h->hist_cur >= 0 ? h->hist[h->hist_cur] : nullptr;
  a.hist_out = h->hist[hout];
  a.cluster = heat1d_impl::async_cluster_size(h->dtype, E, threads, h->S, h->opts.cluster);
  if (a.cluster < 1)
    return fail(HEAT1D_ERR_NOT_RESIDENT, "asynchronous run: clusters of " + std::to_string(h->opts.cluster) +
                                             " CTAs cannot all be resident");
  // empty slots: every word carries version 0x80808080, which no run uses
  HEAT1D_CUDA(cudaMemsetAsync(h->rings, 0x80, 2 * h->esize * h->S * 2 * h->R, h->stream));
  rc = heat1d_impl::launch_async_persistent(a, h->dtype, E, threads, h->stream);
  if (rc == HEAT1D_ERR_NOT_RESIDENT)
    return fail(rc, "asynchronous run: " + std::to_string(h->S) + " CTAs cannot all be resident");
  if (rc) return cuda_fail(cudaGetLastError(), "launch_async_persistent");
  h->cur = 1 - h->cur;
  h->async_step = a.k0 + K;
  h->hist_cur = hout;
  if (out_dev && !out_on_device)
    HEAT1D_CUDA(cudaMemcpyAsync(trace_out, out_dev, tbytes, cudaMemcpyDeviceToHost, h->stream));
  return HEAT1D_OK;
}

// The blocked asynchronous run streamed through HBM: the tiles of the
// streamed synchronous run (W points each, the last one shorter) are the
// segments, Ts steps per block.
int run_blocked_streamed(heat1d* h, int64_t K, uint8_t* trace_out, int out_on_device, const uint8_t* trace_in,
                         int in_on_device) {
  if (h->opts.boundary == 1) return fail(HEAT1D_ERR_INVAL, "streamed runs have Dirichlet ends only");
  if (h->ntiles <= 0 || (h->sE != 4 && h->sE != 8 && h->sE != 16) ||
      h->sthreads > heat1d_impl::kStreamMaxThreads)
    return fail(HEAT1D_ERR_INVAL,
                "streamed run: invalid tile shape (elems_per_thread must be 4, 8 or 16; block_threads at most 512)");
  if (h->snap) return fail(HEAT1D_ERR_INVAL, "snapshots are recorded by on-chip runs only");
  const int64_t nb = (K + h->Ts - 1) / h->Ts;
  if (nb >= INT_MAX) return fail(HEAT1D_ERR_INVAL, "K out of range");
  const size_t sbytes = h->esize * static_cast<size_t>(h->ntiles) * h->R * 2 * h->Th;
  if (sbytes > h->strips_bytes) {
    cudaFree(h->strips);
    h->strips = nullptr;
    h->strips_bytes = 0;
    HEAT1D_CUDA(cudaMalloc(&h->strips, sbytes));
    h->strips_bytes = sbytes;
  }
  const size_t tbytes = static_cast<size_t>(nb) * (h->ntiles - 1) * 2;
  uint8_t* out_dev = nullptr;
  const uint8_t* in_dev = nullptr;
  int rc;
  if ((rc = stage_traces(h, tbytes, trace_out, out_on_device, trace_in, in_on_device, &out_dev, &in_dev))) return rc;
  heat1d_impl::StreamAsyncRun a{};
  a.N = h->N;
  a.K = K;
  a.T = h->Ts;
  a.Th = h->Th;
  a.W = h->W;
  a.ntiles = h->ntiles;
  a.u = h->u[h->cur];  // updated in place
  a.r = h->r;
  a.c1 = h->c1;
  a.cN = h->cN;
  a.q = h->q;
  a.R = h->R;
  a.strips = h->strips;
  a.strips_len = static_cast<int64_t>(h->ntiles) * h->R * 2 * h->Th;
  a.ver = h->done;
  a.trace_out = out_dev;
  a.trace_in = in_dev;
  a.trace_len = static_cast<int64_t>(tbytes);
  a.status = h->status();
  a.spin_limit_ns = h->opts.spin_limit_ns;
  a.stall_tile = h->opts.stall_segment;
  const int resident = heat1d_impl::max_resident_stream_async(h->dtype, h->sE, h->sthreads, h->W + 2 * h->Th);
  if (resident <= 0) return fail(HEAT1D_ERR_NOT_RESIDENT, "streamed asynchronous run: kernel cannot be resident");
  const int grid = static_cast<int>(std::min<int64_t>(h->ntiles, resident));
  if (heat1d_impl::launch_stream_async_setup(a, h->dtype, h->stream))
    return cuda_fail(cudaGetLastError(), "launch_stream_async_setup");
  rc = heat1d_impl::launch_stream_async(a, h->dtype, h->sE, h->sthreads, grid, h->stream);
  if (rc == HEAT1D_ERR_NOT_RESIDENT) return fail(rc, "streamed asynchronous run: grid cannot be resident");
  if (rc) return cuda_fail(cudaGetLastError(), "launch_stream_async");
  if (out_dev && !out_on_device)
    HEAT1D_CUDA(cudaMemcpyAsync(trace_out, out_dev, tbytes, cudaMemcpyDeviceToHost, h->stream));
  return HEAT1D_OK;
}

// The asynchronous run with temporal blocking (blocks of T = h->T steps).
int run_blocked_common(heat1d* h, int64_t K, uint8_t* trace_out, int out_on_device, const uint8_t* trace_in,
                       int in_on_device) {
  if (K < 0 || K >= INT_MAX) return fail(HEAT1D_ERR_INVAL, "K out of range");
  if (K == 0) return HEAT1D_OK;
  reset_history(h);
  if (blocked_streamed(h)) return run_blocked_streamed(h, K, trace_out, out_on_device, trace_in, in_on_device);
  const bool periodic = h->opts.boundary == 1;
  if (periodic && h->S < 2) return fail(HEAT1D_ERR_INVAL, "periodic blocked runs need at least 2 segments");
  int E = 0, threads = 0;
  int rc = pick_shape(h, h->Lmax + 2 * h->T, 0, false, &E, &threads);
  if (rc) return rc;
  if (h->snap) {
    if (K / h->snap_every + 1 > h->snap_rows)
      return fail(HEAT1D_ERR_INVAL, "snapshot buffer holds fewer rows than K/every + 1");
    if (h->snap_every % h->T != 0)
      return fail(HEAT1D_ERR_INVAL, "blocked snapshots need every to be a multiple of the block length");
  }
  const size_t sbytes = h->esize * static_cast<size_t>(h->S) * h->R * 2 * h->T;
  if (sbytes > h->strips_bytes) {
    cudaFree(h->strips);
    h->strips = nullptr;
    h->strips_bytes = 0;
    HEAT1D_CUDA(cudaMalloc(&h->strips, sbytes));
    h->strips_bytes = sbytes;
  }
  const int64_t nb = (K + h->T - 1) / h->T;
  const size_t tbytes = static_cast<size_t>(nb) * (periodic ? h->S : h->S - 1) * 2;
  SegmentRun a = base_run(h, K);
  a.rings = h->strips;
  a.ring_len = h->S * static_cast<int64_t>(h->R) * 2 * h->T;
  uint8_t* out_dev = nullptr;
  const uint8_t* in_dev = nullptr;
  if ((rc = stage_traces(h, tbytes, trace_out, out_on_device, trace_in, in_on_device, &out_dev, &in_dev))) return rc;
  a.trace_out = out_dev;
  a.trace_in = in_dev;
  a.trace_len = static_cast<int64_t>(tbytes);
  a.cluster = heat1d_impl::blocked_cluster_size(h->dtype, E, threads, static_cast<int>(h->S), h->R, h->T,
                                                h->opts.cluster);
  if (a.cluster < 1)
    return fail(HEAT1D_ERR_NOT_RESIDENT, "blocked asynchronous run: clusters of " +
                                             std::to_string(h->opts.cluster) + " CTAs cannot all be resident");
  HEAT1D_CUDA(cudaMemsetAsync(h->prog, 0xff, sizeof(int) * h->S * heat1d_impl::kProgStride, h->stream));
  rc = heat1d_impl::launch_async_blocked(a, h->dtype, E, threads, h->stream);
  if (rc == HEAT1D_ERR_NOT_RESIDENT)
    return fail(rc, "blocked asynchronous run: " + std::to_string(h->S) + " CTAs cannot all be resident");
  if (rc) return cuda_fail(cudaGetLastError(), "launch_async_blocked");
  h->cur = 1 - h->cur;
  if (out_dev && !out_on_device)
    HEAT1D_CUDA(cudaMemcpyAsync(trace_out, out_dev, tbytes, cudaMemcpyDeviceToHost, h->stream));
  return HEAT1D_OK;
}

}  // namespace

extern "C" {

void heat1d_default_opts(heat1d_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->stall_segment = -1;
}

const char* heat1d_last_error(void) { return g_last_error.c_str(); }

heat1d_t heat1d_create(int64_t N, double r, double c1, double cN, int dtype) {
  if (N < 3) {
    fail(HEAT1D_ERR_INVAL, "heat1d_create: N must be >= 3");
    return nullptr;
  }
  if (!(r > 0.0 && r <= 0.5)) {
    fail(HEAT1D_ERR_INVAL, "heat1d_create: r must be in (0, 0.5] (Section 2 stability range)");
    return nullptr;
  }
  if (dtype != HEAT1D_F32 && dtype != HEAT1D_F64) {
    fail(HEAT1D_ERR_INVAL, "heat1d_create: dtype must be HEAT1D_F32 or HEAT1D_F64");
    return nullptr;
  }
  heat1d* h = new heat1d();
  h->N = N;
  h->r = r;
  h->c1 = c1;
  h->cN = cN;
  h->dtype = dtype;
  h->esize = dtype == HEAT1D_F64 ? 8 : 4;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->u[0], h->esize * N);
  if (e == cudaSuccess) e = cudaMalloc(&h->u[1], h->esize * N);
  if (e == cudaSuccess) e = cudaMalloc(&h->ctl, 256);
  if (e == cudaSuccess) e = cudaMemset(h->ctl, 0, 256);
  if (e == cudaSuccess) e = cudaMemset(h->u[0], 0, h->esize * N);
  if (e != cudaSuccess) {
    cuda_fail(e, "heat1d_create");
    heat1d_destroy(h);
    return nullptr;
  }
  heat1d_opts o;
  heat1d_default_opts(&o);
  if (configure(h, o) != HEAT1D_OK) {
    heat1d_destroy(h);
    return nullptr;
  }
  if (h->dtype == HEAT1D_F64)
    set_ends_kernel<double><<<1, 32, 0, h->stream>>>(static_cast<double*>(h->u[0]), N, c1, cN);
  else
    set_ends_kernel<float><<<1, 32, 0, h->stream>>>(static_cast<float*>(h->u[0]), N, c1, cN);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    cuda_fail(e, "heat1d_create");
    heat1d_destroy(h);
    return nullptr;
  }
  return h;
}

void heat1d_destroy(heat1d_t h) {
  if (!h) return;
  free_scratch(h);
  cudaFree(h->u[0]);
  cudaFree(h->u[1]);
  cudaFree(h->ctl);
  cudaFree(h->d_trace);
  delete h;
}

int heat1d_set_snapshots(heat1d_t h, void* buf, int64_t every, int64_t rows) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  if (buf && (every < 1 || rows < 1)) return fail(HEAT1D_ERR_INVAL, "heat1d_set_snapshots: every and rows must be >= 1");
  h->snap = buf;
  h->snap_every = buf ? every : 0;
  h->snap_rows = buf ? rows : 0;
  return HEAT1D_OK;
}

int heat1d_set_stream(heat1d_t h, void* stream) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  h->stream = static_cast<cudaStream_t>(stream);
  return HEAT1D_OK;
}

int heat1d_set_opts(heat1d_t h, const heat1d_opts* o) {
  if (!h || !o) return fail(HEAT1D_ERR_INVAL, "null argument");
  HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
  return configure(h, *o);
}

int heat1d_get_opts(heat1d_t h, heat1d_opts* o) {
  if (!h || !o) return fail(HEAT1D_ERR_INVAL, "null argument");
  *o = h->opts;
  o->segments = h->S;
  o->q = h->q;
  o->halo_steps = h->opts.halo_steps ? h->opts.halo_steps : h->T;
  return HEAT1D_OK;
}

int64_t heat1d_num_segments(heat1d_t h, int64_t* offsets) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  if (offsets) std::memcpy(offsets, h->off.data(), sizeof(int64_t) * (h->S + 1));
  return h->S;
}

int heat1d_set_u(heat1d_t h, const void* u, int on_device) {
  if (!h || !u) return fail(HEAT1D_ERR_INVAL, "null argument");
  reset_history(h);
  HEAT1D_CUDA(cudaMemcpyAsync(h->u[h->cur], u, h->esize * h->N,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  if (h->opts.boundary == 1) {  // periodic: no Dirichlet ends to force
    if (!on_device) HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
    return HEAT1D_OK;
  }
  if (h->dtype == HEAT1D_F64)
    set_ends_kernel<double><<<1, 32, 0, h->stream>>>(static_cast<double*>(h->u[h->cur]), h->N, h->c1, h->cN);
  else
    set_ends_kernel<float><<<1, 32, 0, h->stream>>>(static_cast<float*>(h->u[h->cur]), h->N, h->c1, h->cN);
  HEAT1D_CUDA(cudaGetLastError());
  if (!on_device) HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
  return HEAT1D_OK;
}

int heat1d_get_u(heat1d_t h, void* u, int on_device) {
  if (!h || !u) return fail(HEAT1D_ERR_INVAL, "null argument");
  HEAT1D_CUDA(cudaMemcpyAsync(u, h->u[h->cur], h->esize * h->N,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (!on_device) HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
  return HEAT1D_OK;
}

int heat1d_run_sync(heat1d_t h, int64_t K) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  if (K < 0) return fail(HEAT1D_ERR_INVAL, "K must be >= 0");
  if (K == 0) return HEAT1D_OK;
  reset_history(h);
  int E = 0, threads = 0;
  int rc = h->opts.sync_mode == 2 ? HEAT1D_ERR_INVAL : pick_shape(h, h->Lmax + 2 * h->T, 0, false, &E, &threads);
  if (rc) {
    if (h->opts.sync_mode == 1 || h->opts.boundary == 1) return rc;
    if (h->snap) return fail(HEAT1D_ERR_INVAL, "snapshots are recorded by on-chip runs only");
    return run_streamed(h, K);
  }
  if (h->snap) {
    if (K / h->snap_every + 1 > h->snap_rows)
      return fail(HEAT1D_ERR_INVAL, "snapshot buffer holds fewer rows than K/every + 1");
    if (h->snap_every % h->T != 0)
      return fail(HEAT1D_ERR_INVAL, "synchronous snapshots need every to be a multiple of the halo depth");
  }
  SegmentRun a = base_run(h, K);
  HEAT1D_CUDA(cudaMemsetAsync(h->barrier(), 0, sizeof(unsigned), h->stream));
  rc = heat1d_impl::launch_sync_persistent(a, h->dtype, E, threads, h->stream);
  if (rc == HEAT1D_ERR_NOT_RESIDENT)
    return fail(rc, "synchronous run: " + std::to_string(h->S) + " CTAs cannot all be resident");
  if (rc) return cuda_fail(cudaGetLastError(), "launch_sync_persistent");
  h->cur = 1 - h->cur;
  return HEAT1D_OK;
}

int heat1d_run_async(heat1d_t h, int64_t K, uint8_t* trace_out, int trace_on_device) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  return run_async_common(h, K, trace_out, trace_on_device, nullptr, 0);
}

int heat1d_run_async_blocked(heat1d_t h, int64_t K, uint8_t* trace_out, int trace_on_device) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  return run_blocked_common(h, K, trace_out, trace_on_device, nullptr, 0);
}

int heat1d_replay_blocked(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  if (!trace && h->S > 1 && K > 0) return fail(HEAT1D_ERR_INVAL, "heat1d_replay_blocked: trace is NULL");
  static const uint8_t dummy = 0;
  return run_blocked_common(h, K, nullptr, 0, trace ? trace : &dummy, trace ? trace_on_device : 0);
}

int64_t heat1d_blocked_trace_bytes(heat1d_t h, int64_t K) {
  if (!h || K < 0) return fail(HEAT1D_ERR_INVAL, "bad argument");
  if (blocked_streamed(h)) return (K + h->Ts - 1) / h->Ts * std::max<int64_t>(h->ntiles - 1, 0) * 2;
  return (K + h->T - 1) / h->T * (h->opts.boundary == 1 ? h->S : h->S - 1) * 2;
}

int64_t heat1d_blocked_segments(heat1d_t h, int64_t* offsets, int32_t* block_steps) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  if (!blocked_streamed(h)) {
    if (offsets) std::memcpy(offsets, h->off.data(), sizeof(int64_t) * (h->S + 1));
    if (block_steps) *block_steps = h->T;
    return h->S;
  }
  if (offsets)
    for (int64_t j = 0; j <= h->ntiles; ++j) offsets[j] = std::min<int64_t>(j * h->W, h->N);
  if (block_steps) *block_steps = h->Ts;
  return h->ntiles;
}

int heat1d_async_cluster(heat1d_t h, int blocked) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  int E = 0, threads = 0;
  if (blocked && blocked_streamed(h)) return 1;  // tiles streamed through HBM: no clusters
  const int rc = blocked ? pick_shape(h, h->Lmax + 2 * h->T, 0, false, &E, &threads)
                         : pick_shape(h, h->Lmax + 2, 32 * heat1d_impl::kCommWarps, true, &E, &threads);
  if (rc) return rc;
  const int S = static_cast<int>(h->S);
  const int c = blocked ? heat1d_impl::blocked_cluster_size(h->dtype, E, threads, S, h->R, h->T, h->opts.cluster)
                        : heat1d_impl::async_cluster_size(h->dtype, E, threads, S, h->opts.cluster);
  if (c < 1) return fail(HEAT1D_ERR_NOT_RESIDENT, "clusters of the requested size cannot all be resident");
  return c;
}

int64_t heat1d_trace_bytes(heat1d_t h, int64_t K) {
  if (!h || K < 0) return fail(HEAT1D_ERR_INVAL, "bad argument");
  return K * (h->opts.boundary == 1 ? h->S : h->S - 1) * 2;
}

int heat1d_replay(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  if (!trace && h->S > 1 && K > 0) return fail(HEAT1D_ERR_INVAL, "heat1d_replay: trace is NULL");
  static const uint8_t dummy = 0;
  return run_async_common(h, K, nullptr, 0, trace ? trace : &dummy, trace ? trace_on_device : 0);
}

int64_t heat1d_state_bytes(heat1d_t h) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  return static_cast<int64_t>(sizeof(heat1d_state_header)) +
         static_cast<int64_t>(h->esize) * (h->N + static_cast<int64_t>(h->S) * 2 * h->q);
}

int heat1d_get_state(heat1d_t h, void* state, int on_device) {
  if (!h || !state) return fail(HEAT1D_ERR_INVAL, "null argument");
  heat1d_state_header hd{};
  hd.magic = kStateMagic;
  hd.step = h->hist_cur >= 0 ? h->async_step : 0;
  hd.N = h->N;
  hd.S = h->S;
  hd.q = h->q;
  hd.dtype = h->dtype;
  hd.has_history = h->hist_cur >= 0;
  const size_t ub = h->esize * h->N, hb = h->esize * static_cast<size_t>(h->S) * 2 * h->q;
  void* hist = nullptr;
  if (h->hist_cur >= 0) {
    hist = h->hist[h->hist_cur];
  } else {
    if (hb > h->hist_bytes) {
      cudaFree(h->hist[0]);
      cudaFree(h->hist[1]);
      h->hist[0] = h->hist[1] = nullptr;
      h->hist_bytes = 0;
      HEAT1D_CUDA(cudaMalloc(&h->hist[0], hb));
      HEAT1D_CUDA(cudaMalloc(&h->hist[1], hb));
      h->hist_bytes = hb;
    }
    hist = h->hist[0];
    const int grid = std::min(1024, (h->S + 127) / 128);
    if (h->dtype == HEAT1D_F64)
      edges_history_kernel<double><<<grid, 128, 0, h->stream>>>(static_cast<const double*>(h->u[h->cur]), h->d_off,
                                                                h->S, h->q, static_cast<double*>(hist));
    else
      edges_history_kernel<float><<<grid, 128, 0, h->stream>>>(static_cast<const float*>(h->u[h->cur]), h->d_off,
                                                               h->S, h->q, static_cast<float*>(hist));
    HEAT1D_CUDA(cudaGetLastError());
  }
  unsigned char* out = static_cast<unsigned char*>(state);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (on_device) {
    HEAT1D_CUDA(cudaMemcpyAsync(out, &hd, sizeof(hd), cudaMemcpyHostToDevice, h->stream));
    HEAT1D_CUDA(cudaStreamSynchronize(h->stream));  // hd lives on this stack
  } else {
    std::memcpy(out, &hd, sizeof(hd));
  }
  HEAT1D_CUDA(cudaMemcpyAsync(out + sizeof(hd), h->u[h->cur], ub, kind, h->stream));
  HEAT1D_CUDA(cudaMemcpyAsync(out + sizeof(hd) + ub, hist, hb, kind, h->stream));
  if (!on_device) HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
  return HEAT1D_OK;
}

int heat1d_set_state(heat1d_t h, const void* state, int on_device) {
  if (!h || !state) return fail(HEAT1D_ERR_INVAL, "null argument");
  heat1d_state_header hd{};
  const unsigned char* in = static_cast<const unsigned char*>(state);
  if (on_device) {
    HEAT1D_CUDA(cudaMemcpyAsync(&hd, in, sizeof(hd), cudaMemcpyDeviceToHost, h->stream));
    HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
  } else {
    std::memcpy(&hd, in, sizeof(hd));
  }
  if (hd.magic != kStateMagic) return fail(HEAT1D_ERR_INVAL, "heat1d_set_state: not a heat1d state");
  if (hd.N != h->N || hd.S != h->S || hd.q != h->q || hd.dtype != h->dtype || hd.step < 0)
    return fail(HEAT1D_ERR_INVAL, "heat1d_set_state: the state's N, segments, q or dtype differ from the handle's");
  const size_t ub = h->esize * h->N, hb = h->esize * static_cast<size_t>(h->S) * 2 * h->q;
  if (hb > h->hist_bytes) {
    cudaFree(h->hist[0]);
    cudaFree(h->hist[1]);
    h->hist[0] = h->hist[1] = nullptr;
    h->hist_bytes = 0;
    HEAT1D_CUDA(cudaMalloc(&h->hist[0], hb));
    HEAT1D_CUDA(cudaMalloc(&h->hist[1], hb));
    h->hist_bytes = hb;
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  HEAT1D_CUDA(cudaMemcpyAsync(h->u[h->cur], in + sizeof(hd), ub, kind, h->stream));
  HEAT1D_CUDA(cudaMemcpyAsync(h->hist[0], in + sizeof(hd) + ub, hb, kind, h->stream));
  if (!on_device) HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
  if (hd.has_history) {
    h->hist_cur = 0;
    h->async_step = hd.step;
  } else {
    reset_history(h);
  }
  return HEAT1D_OK;
}

int heat1d_checked(void) { return heat1d_dev::kChecked ? 1 : 0; }

int heat1d_checked_selftest(void) {
  if (!heat1d_dev::kChecked) return fail(HEAT1D_ERR_INVAL, "heat1d_checked_selftest: not a bounds-checked build");
  double* buf = nullptr;
  int* status = nullptr;
  HEAT1D_CUDA(cudaMalloc(&buf, 4 * sizeof(double)));
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
    cudaFree(buf);
    return cuda_fail(cudaGetLastError(), "cudaMalloc(status)");
  }
  int st = 0;
  cudaError_t e = cudaMemset(status, 0, sizeof(int));
  if (e == cudaSuccess) {
    checked_selftest_kernel<<<1, 32>>>(buf, 4, status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  cudaFree(status);
  if (e != cudaSuccess) return cuda_fail(e, "heat1d_checked_selftest");
  return st;
}

int heat1d_sync(heat1d_t h) {
  if (!h) return fail(HEAT1D_ERR_INVAL, "null handle");
  HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
  int st = 0;
  HEAT1D_CUDA(cudaMemcpy(&st, h->status(), sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    HEAT1D_CUDA(cudaMemset(h->status(), 0, sizeof(int)));
    if (st == HEAT1D_ERR_TIMEOUT) return fail(st, "a device-side wait exceeded spin_limit_ns");
    if (st == HEAT1D_ERR_TRACE) return fail(st, "a replay trace entry is >= q");
    if (st == HEAT1D_ERR_BOUNDS) return fail(st, "a kernel index was out of bounds (checked build)");
    return fail(st, "device status " + std::to_string(st));
  }
  return HEAT1D_OK;
}

}  // extern "C"

// ============================================================ batched rods

struct heat1d_batch {
  int dtype = HEAT1D_F64;
  size_t esize = 8;
  int E = 8, threads = 256, grid = 0, T = 16;
  int64_t cap = 0;  // positions per CTA
  int64_t spin_limit_ns = 2000000000LL;
  int stall_slot = -1;  // failure test: this rod part never publishes an epoch
  int64_t nrods = 0, nitems = 0, nparts = 0, counts[3] = {0, 0, 0};
  heat1d_impl::BatchRod* d_rods = nullptr;
  int* d_warp_rods = nullptr;
  heat1d_impl::BatchItem* d_items = nullptr;
  void* d_ctl = nullptr;  // [0]: queue counter, [32]: status word
  int* d_flags = nullptr;
  void* d_edges = nullptr;
  int64_t u_len = 0;  // values of the packed state the rods cover (max offset + N)
  cudaStream_t last_stream = nullptr;
  // asynchronous batched runs (allocated on first use)
  int q = 3, R = 8;
  std::vector<int64_t> part_rod, part_a0, part_L, part_toff;  // per part slot (host)
  std::vector<int64_t> rod_first_slot;                        // per rod: first part slot, -1 if not split
  int64_t trace_bytes = 0;
  int* d_pver = nullptr;
  void* d_strips = nullptr;
  int64_t* d_toff = nullptr;
};

namespace {

void batch_free(heat1d_batch* b) {
  cudaFree(b->d_rods);
  cudaFree(b->d_warp_rods);
  cudaFree(b->d_items);
  cudaFree(b->d_ctl);
  cudaFree(b->d_flags);
  cudaFree(b->d_edges);
  cudaFree(b->d_pver);
  cudaFree(b->d_strips);
  cudaFree(b->d_toff);
}

// Plans the work items: rods that fit one warp window go into warp batches
// (grouped by K so that the warps of a batch finish together), rods that fit
// one CTA become one item, longer rods are split into parts of at most
// cap - 2T points.  Units are queued by decreasing work (points x steps);
// the parts of a rod stay consecutive.
int batch_plan(heat1d_batch* b, const heat1d_rod* rods, int64_t nrods, std::vector<heat1d_impl::BatchRod>& out_rods,
               std::vector<int>& warp_rods, std::vector<heat1d_impl::BatchItem>& items) {
  const int nwarps = b->threads / 32;
  const int64_t warp_cap = 32LL * b->E;
  struct Unit {
    double work;
    int kind;
    int first, count;  // warp batch: range in warp_rods; else rod index
  };
  std::vector<Unit> units;
  std::vector<int> small;
  out_rods.resize(nrods);
  b->rod_first_slot.assign(nrods, -1);
  for (int64_t j = 0; j < nrods; ++j) {
    const heat1d_rod& r = rods[j];
    if (r.N < 3 || r.K < 0 || r.offset < 0 || !(r.r > 0.0 && r.r <= 0.5))
      return fail(HEAT1D_ERR_INVAL, "batched rods: rod " + std::to_string(j) +
                                        " needs N >= 3, K >= 0, offset >= 0 and 0 < r <= 0.5");
    out_rods[j] = heat1d_impl::BatchRod{r.offset, r.N, r.K, r.r, r.c1, r.cN, static_cast<float>(r.r),
                                        static_cast<float>(r.c1), static_cast<float>(r.cN)};
    if (r.K == 0) continue;
    if (r.N <= warp_cap) {
      small.push_back(static_cast<int>(j));
    } else if (r.N <= b->cap) {
      units.push_back(Unit{static_cast<double>(r.N) * r.K, heat1d_impl::kBatchRod, static_cast<int>(j), 1});
    } else {
      units.push_back(Unit{static_cast<double>(r.N) * r.K, heat1d_impl::kBatchPart, static_cast<int>(j), 1});
    }
  }
  std::stable_sort(small.begin(), small.end(), [&](int x, int y) { return rods[x].K > rods[y].K; });
  for (size_t i = 0; i < small.size(); i += nwarps) {
    const int cnt = static_cast<int>(std::min<size_t>(nwarps, small.size() - i));
    double work = 0;
    for (int w = 0; w < cnt; ++w) work += static_cast<double>(rods[small[i + w]].N) * rods[small[i]].K;
    units.push_back(Unit{work, heat1d_impl::kBatchWarps, static_cast<int>(warp_rods.size()), cnt});
    for (int w = 0; w < cnt; ++w) warp_rods.push_back(small[i + w]);
  }
  std::stable_sort(units.begin(), units.end(), [](const Unit& x, const Unit& y) { return x.work > y.work; });
  int slot = 0;
  for (const Unit& un : units) {
    heat1d_impl::BatchItem it{};
    it.kind = un.kind;
    it.rod = un.first;
    it.count = un.count;
    if (un.kind != heat1d_impl::kBatchPart) {
      items.push_back(it);
      b->counts[un.kind] += 1;
      continue;
    }
    const heat1d_rod& r = rods[un.first];
    const int64_t per = b->cap - 2 * b->T;
    const int64_t P = (r.N + per - 1) / per;
    if (P > b->grid)
      return fail(HEAT1D_ERR_INVAL, "batched rods: rod " + std::to_string(un.first) + " needs " + std::to_string(P) +
                                        " CTAs at once, more than can be resident");
    const int64_t base = r.N / P, extra = r.N % P;
    if (base < b->T) return fail(HEAT1D_ERR_INVAL, "batched rods: parts shorter than the halo depth");
    int64_t pos = 0;
    b->rod_first_slot[un.first] = slot;
    const int64_t nblocks = (r.K + b->T - 1) / b->T;
    for (int64_t p = 0; p < P; ++p) {
      const int64_t L = base + (p < extra ? 1 : 0);
      it.part = static_cast<int>(p);
      it.nparts = static_cast<int>(P);
      it.T = b->T;
      it.L = static_cast<int>(L);
      it.slot = slot++;
      it.a0 = pos;
      // an asynchronous run records [ceil(K/T)][2] delays per part
      b->part_rod.push_back(un.first);
      b->part_a0.push_back(pos);
      b->part_L.push_back(L);
      b->part_toff.push_back(b->trace_bytes);
      b->trace_bytes += 2 * nblocks;
      pos += L;
      items.push_back(it);
      b->counts[heat1d_impl::kBatchPart] += 1;
    }
  }
  b->nparts = slot;
  return HEAT1D_OK;
}

}  // namespace

extern "C" {

heat1d_batch_t heat1d_batch_create(const heat1d_rod* rods, int64_t nrods, int dtype, const heat1d_opts* o) {
  if ((!rods && nrods > 0) || nrods < 0) {
    fail(HEAT1D_ERR_INVAL, "heat1d_batch_create: bad rod array");
    return nullptr;
  }
  if (dtype != HEAT1D_F32 && dtype != HEAT1D_F64) {
    fail(HEAT1D_ERR_INVAL, "heat1d_batch_create: dtype must be HEAT1D_F32 or HEAT1D_F64");
    return nullptr;
  }
  heat1d_opts opts;
  heat1d_default_opts(&opts);
  if (o) opts = *o;
  heat1d_batch* b = new heat1d_batch();
  b->dtype = dtype;
  for (int64_t i = 0; i < nrods; ++i) b->u_len = std::max<int64_t>(b->u_len, rods[i].offset + rods[i].N);
  b->esize = dtype == HEAT1D_F64 ? 8 : 4;
  b->E = opts.elems_per_thread ? opts.elems_per_thread : (dtype == HEAT1D_F64 ? 8 : 16);
  b->threads = opts.block_threads ? opts.block_threads : 256;
  b->T = opts.halo_steps ? opts.halo_steps : (dtype == HEAT1D_F64 ? 16 : 32);
  if (opts.spin_limit_ns > 0) b->spin_limit_ns = opts.spin_limit_ns;
  if (opts.q < 0 || opts.q > 255) {
    fail(HEAT1D_ERR_INVAL, "heat1d_batch_create: q must be 1..255 (0: 3)");
    delete b;
    return nullptr;
  }
  b->q = opts.q ? opts.q : 3;
  b->R = 1;
  while (b->R < 2 * b->q) b->R <<= 1;
  b->stall_slot = opts.stall_segment >= 0 && opts.stall_segment < INT_MAX ? static_cast<int>(opts.stall_segment) : -1;
  if ((b->E != 4 && b->E != 8 && b->E != 16 && !(b->E == 32 && b->esize == 4)) || b->threads % 32 != 0 ||
      b->threads < 32 ||
      b->threads > heat1d_impl::max_tile_threads(static_cast<int>(b->esize), b->E) || b->T < 1) {
    fail(HEAT1D_ERR_INVAL, "heat1d_batch_create: elems_per_thread must be 4, 8 or 16 and block_threads a multiple "
                           "of 32 within the CTA limit");
    delete b;
    return nullptr;
  }
  b->cap = heat1d_impl::window_width(b->threads / 32, b->E,
                                     heat1d_impl::sync_window_halo(static_cast<int>(b->esize), b->E));
  if (b->cap - 2 * b->T < b->T) {
    fail(HEAT1D_ERR_INVAL, "heat1d_batch_create: halo_steps too large for the CTA");
    delete b;
    return nullptr;
  }
  b->grid = heat1d_impl::max_resident_batched(dtype, b->E, b->threads);
  if (b->grid <= 0) {
    fail(HEAT1D_ERR_NOT_RESIDENT, "heat1d_batch_create: batched kernel cannot be resident");
    delete b;
    return nullptr;
  }
  std::vector<heat1d_impl::BatchRod> drods;
  std::vector<int> warp_rods;
  std::vector<heat1d_impl::BatchItem> items;
  if (batch_plan(b, rods, nrods, drods, warp_rods, items) != HEAT1D_OK) {
    delete b;
    return nullptr;
  }
  b->nrods = nrods;
  b->nitems = static_cast<int64_t>(items.size());
  b->grid = static_cast<int>(std::min<int64_t>(b->grid, std::max<int64_t>(b->nitems, 1)));
  // a rod's parts must all be resident at once
  for (const auto& it : items)
    if (it.kind == heat1d_impl::kBatchPart && it.nparts > b->grid) b->grid = it.nparts;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(n, 16));
  };
  alloc(reinterpret_cast<void**>(&b->d_rods), sizeof(heat1d_impl::BatchRod) * drods.size());
  alloc(reinterpret_cast<void**>(&b->d_warp_rods), sizeof(int) * warp_rods.size());
  alloc(reinterpret_cast<void**>(&b->d_items), sizeof(heat1d_impl::BatchItem) * items.size());
  alloc(&b->d_ctl, 256);
  alloc(reinterpret_cast<void**>(&b->d_flags), sizeof(int) * b->nparts);
  alloc(&b->d_edges, b->esize * 4 * b->T * std::max<int64_t>(b->nparts, 1));
  if (e == cudaSuccess && !drods.empty())
    e = cudaMemcpy(b->d_rods, drods.data(), sizeof(heat1d_impl::BatchRod) * drods.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !warp_rods.empty())
    e = cudaMemcpy(b->d_warp_rods, warp_rods.data(), sizeof(int) * warp_rods.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(b->d_items, items.data(), sizeof(heat1d_impl::BatchItem) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_ctl, 0, 256);
  if (e != cudaSuccess) {
    cuda_fail(e, "heat1d_batch_create");
    batch_free(b);
    delete b;
    return nullptr;
  }
  return b;
}

namespace {

int batch_run_common(heat1d_batch* b, void* u_packed, void* stream, int async_mode, uint8_t* trace_out,
                     const uint8_t* trace_in) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  b->last_stream = st;
  if (b->nitems == 0) return HEAT1D_OK;
  heat1d_impl::BatchRun a{};
  if (async_mode && b->nparts > 0) {
    if (!b->d_pver) {  // first asynchronous run: version counters, strip rings, trace offsets
      cudaError_t e = cudaMalloc(&b->d_pver, sizeof(int) * b->nparts);
      if (e == cudaSuccess)
        e = cudaMalloc(&b->d_strips, b->esize * static_cast<size_t>(b->nparts) * b->R * 2 * b->T);
      if (e == cudaSuccess) e = cudaMalloc(&b->d_toff, sizeof(int64_t) * b->nparts);
      if (e == cudaSuccess)
        e = cudaMemcpy(b->d_toff, b->part_toff.data(), sizeof(int64_t) * b->nparts, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        cudaFree(b->d_pver);
        cudaFree(b->d_strips);
        cudaFree(b->d_toff);
        b->d_pver = nullptr;
        b->d_strips = nullptr;
        b->d_toff = nullptr;
        return cuda_fail(e, "heat1d_batch: asynchronous buffers");
      }
    }
    a.async_mode = async_mode;
    a.q = b->q;
    a.R = b->R;
    a.pver = b->d_pver;
    a.strips = b->d_strips;
    a.toff = b->d_toff;
    a.trace_out = trace_out;
    a.trace_in = trace_in;
    a.strips_len = static_cast<int64_t>(b->nparts) * b->R * 2 * b->T;
    a.trace_len = b->trace_bytes;
    HEAT1D_CUDA(cudaMemsetAsync(b->d_pver, 0xff, sizeof(int) * b->nparts, st));
  }
  a.rods = b->d_rods;
  a.warp_rods = b->d_warp_rods;
  a.items = b->d_items;
  a.nitems = b->nitems;
  a.u = u_packed;
  a.counter = static_cast<unsigned*>(b->d_ctl);
  a.flags = b->d_flags;
  a.edges = b->d_edges;
  a.u_len = b->u_len;
  a.edges_len = 4 * static_cast<int64_t>(b->T) * std::max<int64_t>(b->nparts, 1);
  a.Tmax = b->T;
  a.one = 1.0;
  a.one_f = 1.0f;
  a.status = static_cast<int*>(b->d_ctl) + 32;
  a.spin_limit_ns = b->spin_limit_ns;
  a.stall_slot = b->stall_slot;
  HEAT1D_CUDA(cudaMemsetAsync(b->d_ctl, 0, sizeof(unsigned), st));
  if (b->nparts > 0) HEAT1D_CUDA(cudaMemsetAsync(b->d_flags, 0, sizeof(int) * b->nparts, st));
  int rc = heat1d_impl::launch_batched(a, b->dtype, b->E, b->threads, b->grid, st);
  if (rc == HEAT1D_ERR_NOT_RESIDENT) return fail(rc, "heat1d_batch_run: grid cannot be resident");
  if (rc) return cuda_fail(cudaGetLastError(), "launch_batched");
  return HEAT1D_OK;
}

}  // namespace

int heat1d_batch_run(heat1d_batch_t b, void* u_packed, void* stream) {
  if (!b || !u_packed) return fail(HEAT1D_ERR_INVAL, "heat1d_batch_run: null argument");
  return batch_run_common(b, u_packed, stream, 0, nullptr, nullptr);
}

int heat1d_batch_run_async(heat1d_batch_t b, void* u_packed, void* stream, uint8_t* trace_out) {
  if (!b || !u_packed) return fail(HEAT1D_ERR_INVAL, "heat1d_batch_run_async: null argument");
  return batch_run_common(b, u_packed, stream, 1, trace_out, nullptr);
}

int heat1d_batch_replay(heat1d_batch_t b, void* u_packed, void* stream, const uint8_t* trace) {
  if (!b || !u_packed) return fail(HEAT1D_ERR_INVAL, "heat1d_batch_replay: null argument");
  if (!trace && b->nparts > 0) return fail(HEAT1D_ERR_INVAL, "heat1d_batch_replay: trace is NULL");
  return batch_run_common(b, u_packed, stream, 2, nullptr, trace);
}

int64_t heat1d_batch_trace_bytes(heat1d_batch_t b) {
  if (!b) return fail(HEAT1D_ERR_INVAL, "null batch");
  return b->trace_bytes;
}

int64_t heat1d_batch_rod_parts(heat1d_batch_t b, int64_t rod, int64_t* offsets, int64_t* trace_offset) {
  if (!b || rod < 0 || rod >= b->nrods) return fail(HEAT1D_ERR_INVAL, "heat1d_batch_rod_parts: bad argument");
  const int64_t first = b->rod_first_slot[rod];
  if (first < 0) {
    if (trace_offset) *trace_offset = -1;
    return 1;
  }
  int64_t P = 0;
  while (first + P < b->nparts && b->part_rod[first + P] == rod) ++P;
  if (offsets) {
    for (int64_t p = 0; p < P; ++p) offsets[p] = b->part_a0[first + p];
    offsets[P] = b->part_a0[first + P - 1] + b->part_L[first + P - 1];
  }
  if (trace_offset) *trace_offset = b->part_toff[first];
  return P;
}

int heat1d_batch_sync(heat1d_batch_t b) {
  if (!b) return fail(HEAT1D_ERR_INVAL, "null batch");
  HEAT1D_CUDA(cudaStreamSynchronize(b->last_stream));
  int st = 0;
  HEAT1D_CUDA(cudaMemcpy(&st, static_cast<int*>(b->d_ctl) + 32, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    HEAT1D_CUDA(cudaMemset(static_cast<int*>(b->d_ctl) + 32, 0, sizeof(int)));
    return fail(st, st == HEAT1D_ERR_TIMEOUT  ? "a device-side wait exceeded spin_limit_ns"
                    : st == HEAT1D_ERR_BOUNDS ? "a kernel index was out of bounds (checked build)"
                                              : "device status " + std::to_string(st));
  }
  return HEAT1D_OK;
}

int heat1d_batch_describe(heat1d_batch_t b, int64_t* info) {
  if (!b || !info) return fail(HEAT1D_ERR_INVAL, "null argument");
  info[0] = b->counts[heat1d_impl::kBatchWarps];
  info[1] = b->counts[heat1d_impl::kBatchRod];
  info[2] = b->counts[heat1d_impl::kBatchPart];
  info[3] = b->grid;
  info[4] = b->threads;
  info[5] = b->E;
  info[6] = b->T;
  info[7] = b->cap;
  return HEAT1D_OK;
}

void heat1d_batch_destroy(heat1d_batch_t b) {
  if (!b) return;
  batch_free(b);
  delete b;
}

int heat1d_run_batched(const heat1d_rod* rods, int64_t nrods, void* u_packed, int dtype, const heat1d_opts* o,
                       void* stream) {
  heat1d_batch_t b = heat1d_batch_create(rods, nrods, dtype, o);
  if (!b) return g_last_error.find("resident") != std::string::npos ? HEAT1D_ERR_NOT_RESIDENT : HEAT1D_ERR_INVAL;
  int rc = heat1d_batch_run(b, u_packed, stream);
  if (rc == HEAT1D_OK) rc = heat1d_batch_sync(b);
  heat1d_batch_destroy(b);
  return rc;
}

}  // extern "C"

// ============================================================ adjoint

extern "C" {

static int adjoint_handle(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device, const double* u_obs,
                          int cotangent, int64_t ckpt_every, double* grad_u0, double* grad_r, double* loss) {
  if (!h || !u_obs || !grad_u0) return fail(HEAT1D_ERR_INVAL, "heat1d_adjoint: null argument");
  if (h->opts.boundary == 1) return fail(HEAT1D_ERR_INVAL, "heat1d_adjoint: Dirichlet ends only");
  if (K < 0) return fail(HEAT1D_ERR_INVAL, "heat1d_adjoint: K must be >= 0");
  const bool async_run = trace != nullptr && h->S > 1;
  const size_t tbytes = static_cast<size_t>(K) * (h->S - 1) * 2;
  const uint8_t* dtrace = nullptr;
  int rc;
  if (async_run) {
    if (trace_on_device) {
      dtrace = trace;
    } else {
      if ((rc = ensure_trace_staging(h, tbytes))) return rc;
      HEAT1D_CUDA(cudaMemcpyAsync(h->d_trace, trace, tbytes, cudaMemcpyHostToDevice, h->stream));
      dtrace = h->d_trace;
    }
  }
  // host-side check of the trace window (the kernels assume every d < q)
  if (async_run) {
    std::vector<uint8_t> tr(tbytes);
    HEAT1D_CUDA(cudaMemcpyAsync(tr.data(), dtrace, tbytes, cudaMemcpyDeviceToHost, h->stream));
    HEAT1D_CUDA(cudaStreamSynchronize(h->stream));
    for (size_t j = 0; j < tbytes; ++j)
      if (tr[j] >= h->q) return fail(HEAT1D_ERR_TRACE, "heat1d_adjoint: trace entry >= q");
  }
  heat1d_impl::AdjointRun a{};
  a.nrods = 1;
  a.N = h->N;
  a.K = K;
  a.r = &h->r;
  a.c1 = &h->c1;
  a.cN = &h->cN;
  a.S = h->S;
  a.q = h->q;
  a.trace = dtrace;
  a.u0 = h->u[h->cur];
  a.u_obs = u_obs;
  a.ckpt_every = ckpt_every > 0 ? ckpt_every : 128;
  a.uK = h->u[1 - h->cur];
  a.grad_u0 = grad_u0;
  a.grad_r = grad_r;
  a.loss = loss;
  a.cotangent = cotangent;
  a.stream = h->stream;
  rc = heat1d_impl::run_adjoint(a, h->dtype);
  if (rc == HEAT1D_ERR_OOM) return fail(rc, "heat1d_adjoint: out of device memory for checkpoints");
  if (rc) return cuda_fail(cudaGetLastError(), "heat1d_adjoint");
  h->cur = 1 - h->cur;  // the state is now u(K)
  reset_history(h);
  return HEAT1D_OK;
}

int heat1d_adjoint(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device, const double* u_obs,
                   int64_t ckpt_every, double* grad_u0, double* grad_r, double* loss) {
  return adjoint_handle(h, K, trace, trace_on_device, u_obs, 0, ckpt_every, grad_u0, grad_r, loss);
}

int heat1d_vjp(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device, const double* grad_uK,
               int64_t ckpt_every, double* grad_u0, double* grad_r) {
  return adjoint_handle(h, K, trace, trace_on_device, grad_uK, 1, ckpt_every, grad_u0, grad_r, nullptr);
}

int heat1d_adjoint_batched(int64_t nrods, int64_t N, int64_t K, const double* r, const double* c1, const double* cN,
                           int dtype, const void* u0, const double* u_obs, int cotangent, int64_t segments, int q,
                           const uint8_t* trace, int64_t ckpt_every, void* uK, double* grad_u0, double* grad_r,
                           double* loss, void* stream) {
  if (nrods < 1 || N < 3 || K < 0 || !r || !c1 || !cN || !u0 || !u_obs || !grad_u0)
    return fail(HEAT1D_ERR_INVAL, "heat1d_adjoint_batched: bad argument");
  if (dtype != HEAT1D_F32 && dtype != HEAT1D_F64) return fail(HEAT1D_ERR_INVAL, "heat1d_adjoint_batched: dtype");
  for (int64_t j = 0; j < nrods; ++j)
    if (!(r[j] > 0.0 && r[j] <= 0.5)) return fail(HEAT1D_ERR_INVAL, "heat1d_adjoint_batched: r out of (0, 0.5]");
  if (trace && (segments < 2 || segments > N || q < 1 || q > 255))
    return fail(HEAT1D_ERR_INVAL, "heat1d_adjoint_batched: a trace needs 2 <= segments <= N and 1 <= q <= 255");
  heat1d_impl::AdjointRun a{};
  a.nrods = nrods;
  a.N = N;
  a.K = K;
  a.r = r;
  a.c1 = c1;
  a.cN = cN;
  a.S = trace ? static_cast<int>(segments) : 1;
  a.q = trace ? q : 1;
  a.trace = trace;
  a.u0 = u0;
  a.u_obs = u_obs;
  a.ckpt_every = ckpt_every > 0 ? ckpt_every : 128;
  a.uK = uK;
  a.grad_u0 = grad_u0;
  a.grad_r = grad_r;
  a.loss = loss;
  a.cotangent = cotangent;
  a.stream = static_cast<cudaStream_t>(stream);
  int rc = heat1d_impl::run_adjoint(a, dtype);
  if (rc == HEAT1D_ERR_OOM) return fail(rc, "heat1d_adjoint_batched: out of device memory for checkpoints");
  if (rc) return cuda_fail(cudaGetLastError(), "heat1d_adjoint_batched");
  return HEAT1D_OK;
}

}  // extern "C"

// noalloc_api.cu -- heat1d_run_sync_noalloc: the synchronous run for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs where allocation is not
// allowed or not safe, such as a host callback, a custom allocator's own
// hooks, a plug-in that must not grow the process's device footprint, or a
// real-time loop that forbids allocation after start-up.  The handle API
// allocates its state and scratch when a handle is created, so it is not open
// to them.  This entry point takes the caller's input and output buffers and
// keeps the synchronous kernel's scratch (the halo exchange buffers, the grid
// barrier counter, the status word and the segment offsets) in one file-scope
// __device__ array of fixed size.  Every GPU that loads the library holds that
// array until the process exits.
#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>  // CUcontext and the driver's function types only; nothing is linked from libcuda
#include <cuda_runtime.h>

#include "heat1d.h"
#include "impl.h"

namespace {

// Limits of the shared scratch array.  The halo buffers hold kNoallocHaloBytes
// per segment side and parity: 128 FP32 or 64 FP64 points, the handle API's
// default halo depths.
constexpr int kNoallocMaxSegments = 256;
constexpr int kNoallocHaloBytes = 512;
// Layout (bytes): [0, 256) control words (barrier counter at 0, status at 128);
// [256, 256 + 8*(S+1)) segment offsets; then the halo buffers [2][S][2T] values.
constexpr size_t kCtlBytes = 256;
constexpr size_t kOffBytes = 8 * (kNoallocMaxSegments + 1);
constexpr size_t kEdgeOffset = (kCtlBytes + kOffBytes + 255) / 256 * 256;
constexpr size_t kEdgeBytes = size_t(2) * kNoallocMaxSegments * 2 * kNoallocHaloBytes;
constexpr size_t kScratchBytes = kEdgeOffset + kEdgeBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The array's device address is valid in the CUDA context in which it was
// looked up; it is cached per context, keyed by the context's unique id (ids
// are never reused within a process, so a context destroyed by a device reset
// and a later one at the same handle value are told apart).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
struct ScratchEntry {
  unsigned long long ctx_id;
  void* addr;
};
std::mutex g_mu;
std::vector<ScratchEntry> g_scratch;  // grows by one entry per context; reserved up front
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Clears the control words and writes the segment offsets (the first N mod S
// segments hold one point more), so that nothing depends on an earlier call.
__global__ void noalloc_prepare_kernel(unsigned char* scratch, int64_t N, int S) {
  unsigned* barrier = reinterpret_cast<unsigned*>(scratch);
  int* status = reinterpret_cast<int*>(scratch + 128);
  int64_t* off = reinterpret_cast<int64_t*>(scratch + kCtlBytes);
  const int64_t base = N / S, extra = N % S;
  for (int s = threadIdx.x; s <= S; s += blockDim.x) off[s] = s * base + (s < extra ? s : extra);
  if (threadIdx.x == 0) {
    *barrier = 0u;
    *status = 0;
  }
}

// Copies the run's device status to the caller's word.
__global__ void noalloc_status_kernel(const unsigned char* scratch, int* status_out) {
  if (threadIdx.x == 0) *status_out = *reinterpret_cast<const int*>(scratch + 128);
}

int fail(int code, const std::string& msg) {
  heat1d_impl::set_last_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(HEAT1D_ERR_CUDA, std::string("heat1d_run_sync_noalloc: ") + what + ": " + cudaGetErrorString(e));
}

// Looks up the scratch array's device address in the calling thread's current
// context (the current device's primary context unless the caller made
// another one current), once per context.
int scratch_address(int dev, unsigned char** out) {
  // Makes the device's primary context current on this thread and
  // initialises it if needed (a no-op when the caller already uses it).
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    void* f1 = nullptr;
    void* f2 = nullptr;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f1)
      return fail(HEAT1D_ERR_CUDA, "heat1d_run_sync_noalloc: driver entry point cuCtxGetCurrent not found");
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !f2)
      return fail(HEAT1D_ERR_CUDA, "heat1d_run_sync_noalloc: driver entry point cuCtxGetId not found");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    g_scratch.reserve(64);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_get_id(ctx, &id) != CUDA_SUCCESS)
    return fail(HEAT1D_ERR_CUDA, "heat1d_run_sync_noalloc: no current CUDA context");
  for (const ScratchEntry& s : g_scratch) {
    if (s.ctx_id == id) {
      *out = static_cast<unsigned char*>(s.addr);
      return HEAT1D_OK;
    }
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress");
  g_scratch.push_back({id, p});
  *out = static_cast<unsigned char*>(p);
  return HEAT1D_OK;
}

}  // namespace

extern "C" int heat1d_run_sync_noalloc(const void* u_in, void* u_out, int64_t N, double r, double c1, double cN,
                                       int dtype, int64_t K, int64_t segments, void* stream, int* status_out) {
  if (!u_in || !u_out) return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: null buffer");
  if (u_in == u_out) return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: u_in and u_out must differ");
  if (N < 3) return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: N must be >= 3");
  if (!(r > 0.0 && r <= 0.5)) return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: r must be in (0, 0.5]");
  if (dtype != HEAT1D_F32 && dtype != HEAT1D_F64)
    return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: dtype must be HEAT1D_F32 or HEAT1D_F64");
  if (K < 0) return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: K must be >= 0");
  if (segments < 0 || segments > kNoallocMaxSegments)
    return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: segments must be in [0, 256] (the size of the "
                                  "library's fixed scratch array)");

  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (nsm < 1) return fail(HEAT1D_ERR_CUDA, "heat1d_run_sync_noalloc: device reports no multiprocessors");

  unsigned char* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc) return rc;

  int64_t S = segments ? segments : std::min<int64_t>(nsm, kNoallocMaxSegments);
  S = std::min<int64_t>(S, N);
  if (S < 1) return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: no segments");
  const int64_t Lmin = N / S, Lmax = N / S + (N % S ? 1 : 0);
  const int esize = dtype == HEAT1D_F64 ? 8 : 4;
  // The handle API's default halo depth capped at what the array holds (FP32
  // 128 steps; FP64 64 on segments of 4096 points or more, else 32), at most
  // the shortest segment.  The depth changes the speed, never the result.
  const int Tdef = esize == 4 ? 128 : (Lmin >= 4096 ? 64 : 32);
  const int T = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(Tdef, Lmin)));
  static_assert(kNoallocHaloBytes >= 128 * 4 && kNoallocHaloBytes >= 64 * 8, "halo buffers too small");

  // Launch shape: the handle API's rule -- the fewest points per thread that
  // fit one CTA, FP32 trying 16 points per thread first on tiles of at least
  // 8 warps of 16 points.
  const int64_t slots = Lmax + 2 * T;
  const bool prefer16 = esize == 4 && slots >= 8 * 32 * 16;
  const int Es[4] = {2, 4, 8, 16};
  const int Es16[4] = {16, 2, 4, 8};
  int E = 0, threads = 0;
  for (int i = 0; i < 4 && !E; ++i) {
    const int e = prefer16 ? Es16[i] : Es[i];
    const int64_t t = 32 * heat1d_impl::window_warps(slots, e, heat1d_impl::sync_window_halo(esize, e));
    if (t <= heat1d_impl::max_tile_threads(esize, e)) {
      E = e;
      threads = static_cast<int>(t);
    }
  }
  if (!E)
    return fail(HEAT1D_ERR_INVAL, "heat1d_run_sync_noalloc: " + std::to_string(Lmax) +
                                      " points per segment exceed one CTA; pass more segments (at most 256)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  noalloc_prepare_kernel<<<1, 256, 0, st>>>(scratch, N, static_cast<int>(S));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "prepare");

  {
    // K = 0 still launches: the kernel then only copies u(0), ends forced.
    heat1d_impl::SegmentRun a{};
    a.N = N;
    a.K = K;
    a.S = static_cast<int>(S);
    a.seg_off = reinterpret_cast<const int64_t*>(scratch + kCtlBytes);
    a.u_in = u_in;
    a.u_out = u_out;
    a.r = r;
    a.c1 = c1;
    a.cN = cN;
    a.status = reinterpret_cast<int*>(scratch + 128);
    a.spin_limit_ns = 2000000000LL;
    a.T = T;
    a.edges = scratch + kEdgeOffset;
    a.edges_len = 2 * S * 2 * static_cast<int64_t>(T);
    a.barrier = reinterpret_cast<unsigned*>(scratch);
    a.stall_segment = -1;
    rc = heat1d_impl::launch_sync_persistent(a, dtype, E, threads, st);
    if (rc == HEAT1D_ERR_NOT_RESIDENT)
      return fail(rc, "heat1d_run_sync_noalloc: " + std::to_string(S) + " CTAs cannot all be resident");
    if (rc) return cuda_fail(cudaGetLastError(), "launch");
  }
  if (status_out) {
    noalloc_status_kernel<<<1, 32, 0, st>>>(scratch, status_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "status");
  }
  return HEAT1D_OK;
}

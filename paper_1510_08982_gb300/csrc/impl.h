// impl.h -- internal interface between the C ABI (heat1d_api.cu) and the
// kernel translation units.  Not installed; not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace heat1d_impl {

// Largest ring of the asynchronous run (versions kept per directed edge).
constexpr int kMaxRing = 512;
// Communication warps per CTA of the asynchronous kernel (left puller, right
// puller).
constexpr int kCommWarps = 2;
// Padding, in ints, between the per-segment version counters (one 128-byte
// line each, so that CTAs never share a line they write).
constexpr int kProgStride = 32;

// Arguments of one persistent run over the segments of one rod.
struct SegmentRun {
  int64_t N;
  int64_t K;
  int S;
  const int64_t* seg_off;  // device, S+1 offsets
  const void* u_in;        // device, N values
  void* u_out;             // device, N values (a different buffer)
  double r, c1, cN;
  float r_f, c1_f, cN_f;   // the same rounded to float (FP32 runs; set at launch)
  double one;              // 1.0 as a run-time value (see ftcs in common.cuh); one_f its float
  float one_f;
  int* status;             // device status word (0 = healthy)
  int64_t spin_limit_ns;
  int periodic;            // 1: periodic ring (Section 5.3), no Dirichlet ends
  void* snap;              // device [K/snap_every + 1][N] states at steps j*snap_every, or null
  int64_t snap_every;

  // synchronous run
  int T;                   // halo width = steps between exchanges
  void* edges;             // [2][S][2T] values
  unsigned* barrier;       // grid barrier counter, zero at launch

  // asynchronous run / replay
  int q;                   // delay window
  int R;                   // ring length (power of two, >= 2q)
  int* prog;               // blocked run: [S * kProgStride] strip versions, -1 at launch
  void* rings;             // per-step run: [S][2][R][sizeof(real)/4] tagged slot words (uint64, version in
                           // the high half, 32 value bits in the low half), cleared to bytes 0x80;
                           // [s][0] the first point, [s][1] the last point.  Blocked run: the strips.
  uint8_t* trace_out;      // device or NULL
  const uint8_t* trace_in; // device, replay only
  int stall_segment;       // -1: off
  // Resuming an asynchronous run (checkpoint/restart): the run's step 0 is
  // global step k0 of a longer run; hist_in (device [S][2][q], or NULL when
  // k0 = 0) holds every segment's first and last point at global steps
  // k0-q+1 .. k0 (oldest first), the versions a step may still read; the run
  // writes the same for its own last q steps to hist_out (device, or NULL).
  int64_t k0;
  const void* hist_in;
  void* hist_out;
  // CTAs per thread-block cluster (1: none).  Neighbouring segments in one
  // cluster hand their edge values to each other through distributed shared
  // memory; the others through the global rings.
  int cluster;
  // Buffer extents, in elements, for the bounds-checked build (checked.cuh):
  // snapshots, trace (bytes), rings or strips, edges, edge histories.
  int64_t snap_len, trace_len, ring_len, edges_len, hist_len;
};

// Arguments of one temporally blocked synchronous run streamed through HBM.
struct StreamRun {
  int64_t N;
  int64_t K;
  int T;                   // steps per pass
  int Th;                  // halo points loaded per side (>= T, 16-byte multiple)
  int W;                   // tile width (points written per tile), 16-byte multiple
  int64_t ntiles;
  void* u_a;               // state at pass 0 (read), then alternating
  void* u_b;
  double r, c1, cN;
  float r_f, c1_f, cN_f;   // FP32 copies and the run-time 1.0, as in SegmentRun
  double one;
  float one_f;
  int* done;               // [ntiles] passes completed per tile, 0 at launch
  int* status;
  int64_t spin_limit_ns;
  int64_t stall_tile;      // -1: off; else that tile never publishes a pass (failure test)
};

// Largest CTA (threads) of the register-tile kernels for a dtype and E: a
// tile of more than 64 bytes per thread needs more than 64 registers per
// thread, so it is limited to 512 threads (up to 128 registers).  So is the
// FP32 tile of 16 points: its two register arrays of 16 floats and the loop
// state did not fit 64 registers (ptxas spilled 112-324 bytes per thread in
// the synchronous and batched kernels).
// The FP32 tile of 32 points (two arrays of 32 floats) is limited to 256
// threads, so that it may use up to 255 registers.
constexpr int max_tile_threads(int elem_bytes, int E) {
  return (elem_bytes == 4 && E == 32) ? 256 : ((elem_bytes * E > 64 || (elem_bytes == 4 && E == 16)) ? 512 : 1024);
}
// The asynchronous kernel adds its communication warps to the compute
// threads (within the 1024-thread CTA limit).
constexpr int max_async_threads(int elem_bytes, int E) {
  return max_tile_threads(elem_bytes, E) + 32 * kCommWarps > 1024 ? 1024 : max_tile_threads(elem_bytes, E) + 32 * kCommWarps;
}

// Warp windows (common.cuh): warp w covers 32E positions starting at w*D,
// D = 32E - 2H, where H (halo points per warp side = steps between two
// refreshes) trades redundant arithmetic (2H/32E) against barriers (one per
// H steps).  The synchronous kernels use H = E/2 in FP32 (H = E for E = 16
// on chip) and E/4 in FP64 (at least 1): FP64 arithmetic is costly, so less
// redundancy is worth more barriers.  The asynchronous kernel uses H = E/2: its edge warps must not be
// held back by frequent barriers.  A CTA of nw compute warps covers
// nw*D + 2H positions.
// FP32 tiles take H = E/2.  Whole-lane halos (H = E = 16: lanes 0 and 31 the
// halos, refreshed every 16 steps; Window allows the form) were measured on
// GB300 and lost: 4.75e12 against 7.33e12 updates/s on the 2^20-point rod at
// T = 512, 0.33 against 0.41 of the FP32 ALU roofline on the uneven batch.
constexpr int sync_window_halo(int elem_bytes, int E) { return elem_bytes == 8 ? (E >= 4 ? E / 4 : 1) : E / 2; }
constexpr int stream_window_halo(int elem_bytes, int E) { return elem_bytes == 8 ? (E >= 4 ? E / 4 : 1) : E / 2; }
constexpr int async_window_halo(int /*elem_bytes*/, int E) { return E / 2; }
constexpr int64_t window_width(int64_t nwarps, int E, int H) { return nwarps * (32 * E - 2 * H) + 2 * H; }
constexpr int64_t window_warps(int64_t positions, int E, int H) {
  return positions <= 2 * H ? 1 : (positions - 2 * H + (32 * E - 2 * H) - 1) / (32 * E - 2 * H);
}

// Sets the FP32 copies of a run's parameters (round to nearest, as a device
// conversion would) and the run-time 1.0.  Every launch function applies it
// to its copy of the arguments.
template <typename Run>
inline void set_run_params(Run& a) {
  a.r_f = static_cast<float>(a.r);
  a.c1_f = static_cast<float>(a.c1);
  a.cN_f = static_cast<float>(a.cN);
  a.one = 1.0;
  a.one_f = 1.0f;
}

// Launch the persistent kernels (cooperative launch: all S CTAs resident).
// E is the number of points per thread (2, 4, 8 or 16); `threads` the compute
// threads per CTA (a multiple of 32).  Return a heat1d_status code.
int launch_sync_persistent(const SegmentRun& a, int dtype, int E, int threads, cudaStream_t st);
int launch_async_persistent(const SegmentRun& a, int dtype, int E, int threads, cudaStream_t st);
// Cluster size for the asynchronous per-step run of S segments: `wanted` 0
// picks the largest of 8, 4, 2 that divides S with every cluster resident
// (else 1); 1, 2, 4 or 8 is checked.  Returns 0 when `wanted` cannot be met.
int async_cluster_size(int dtype, int E, int threads, int S, int wanted);
// Asynchronous run with temporal blocking: a.T steps per block, a.rings holds
// [S][R][2T] strips, a.prog the per-segment strip versions (-1 at launch).
int launch_async_blocked(const SegmentRun& a, int dtype, int E, int threads, cudaStream_t st);
// Cluster size for the blocked run (as async_cluster_size; a cluster launch
// keeps the neighbours' strip rings, 2*R*T values, in shared memory, at most
// kMaxClusterStripBytes).
constexpr size_t kMaxClusterStripBytes = 96 * 1024;
int blocked_cluster_size(int dtype, int E, int threads, int S, int R, int T, int wanted);

// Sets the message returned by heat1d_last_error() on this host thread.
void set_last_error(const std::string& msg);

// Streamed synchronous run: one cooperative launch of `grid` CTAs of `threads`
// compute threads (at most kStreamMaxThreads) plus a loader and a releaser
// warp, E points per thread (4, 8 or 16); tile loads by bulk copies into
// shared memory.
constexpr int kStreamMaxThreads = 512;
int launch_stream_tma(const StreamRun& a, int dtype, int E, int threads, int grid, cudaStream_t st);
int max_resident_stream_tma(int dtype, int E, int threads, int Wt);

// Arguments of one asynchronous run with temporal blocking streamed through
// HBM: the tiles are the segments of the blocked model (tile j = points
// [jW, min((j+1)W, N))), each advanced T steps per block on its own points
// and two halo strips taken from its neighbours' published versions.
struct StreamAsyncRun {
  int64_t N;
  int64_t K;
  int T;                   // steps per block
  int Th;                  // halo points kept per side (>= T, 16-byte multiple)
  int W;                   // tile width, 16-byte multiple
  int64_t ntiles;
  void* u;                 // state, updated in place (each tile reads and writes only its own points)
  double r, c1, cN;
  float r_f, c1_f, cN_f;   // FP32 copies and the run-time 1.0, as in SegmentRun
  double one;
  float one_f;
  int q;                   // delay window in blocks
  int R;                   // strip versions kept per tile (power of two, >= 2q)
  void* strips;            // [ntiles][R][2*Th]: first Th and last Th points of a tile per version
  int* ver;                // [ntiles] newest version published (set to 0 by the set-up kernel)
  uint8_t* trace_out;      // device [ceil(K/T)][ntiles-1][2] or NULL
  const uint8_t* trace_in; // replay: device, same layout
  int* status;
  int64_t spin_limit_ns;
  int64_t stall_tile;      // -1: off; else that tile never publishes (failure test)
  int64_t strips_len, trace_len;  // extents in elements / bytes (bounds-checked build)
};
// Publishes version 0 of every tile's strips (the initial state) and sets the
// version counters to 0; then the persistent launch (cooperative, `grid` CTAs
// of `threads` compute threads plus a loader and a releaser warp).
int launch_stream_async_setup(const StreamAsyncRun& a, int dtype, cudaStream_t st);
int launch_stream_async(const StreamAsyncRun& a, int dtype, int E, int threads, int grid, cudaStream_t st);
int max_resident_stream_async(int dtype, int E, int threads, int Wt);

// ------------------------------------------------------------ batched rods

// One rod of a batch as the kernels see it.
struct BatchRod {
  int64_t offset;  // first point in the packed state
  int64_t N;
  int64_t K;
  double r, c1, cN;
  float r_f, c1_f, cN_f;  // the same rounded to float (FP32 batches)
};

// One work item: what one CTA does between two grabs from the queue.
enum BatchKind { kBatchWarps = 0, kBatchRod = 1, kBatchPart = 2 };
struct BatchItem {
  int kind;    // BatchKind
  int rod;     // kBatchWarps: first entry in warp_rods; else the rod
  int count;   // kBatchWarps: rods in the batch (one per warp)
  int part;    // kBatchPart: index of the part in the rod, and of its parts
  int nparts;
  int T;       // kBatchPart: halo depth = steps between exchanges
  int L;       // kBatchPart: points of the part
  int slot;    // kBatchPart: index of the part's flag and edge buffers
  int64_t a0;  // kBatchPart: first point of the part (rod-relative)
};

struct BatchRun {
  const BatchRod* rods;
  const int* warp_rods;   // rods of the warp batches, in batch order
  const BatchItem* items;
  int64_t nitems;
  void* u;                // packed state, updated in place
  unsigned* counter;      // queue position, zero at launch
  int* flags;             // per part: 1 after loading, e+2 after publishing epoch e; zero at launch
  void* edges;            // per part: [2 parities][2][Tmax] values
  int Tmax;
  double one;             // 1.0 as a run-time value; one_f its float
  float one_f;
  int* status;
  int64_t spin_limit_ns;
  int stall_slot;         // -1: off; else the part in that flag slot never publishes an epoch (failure test)
  int64_t u_len, edges_len;  // extents of u and edges in elements (bounds-checked build)
  // Asynchronous batched run: the parts of each split rod are the segments of
  // the blocked model (Eq. (eqn:async) per block of T steps, strips up to q-1
  // blocks old); rods that fit one CTA or one warp have no inner boundary and
  // run as above.
  int async_mode;          // 0: synchronous; 1: free run (trace recorded); 2: replay of trace_in
  int q, R;                // delay window in blocks; strip versions kept per part (power of two >= 2q)
  int* pver;               // [nparts] newest strip version published, -1 at launch
  void* strips;            // [nparts][R][2][Tmax] values: first and last T points of a part per version
  const int64_t* toff;     // [nparts] byte offset of each part's trace: [ceil(K/T)][2], [j][0] the left read
  uint8_t* trace_out;      // free run: delays, or null
  const uint8_t* trace_in; // replay
  int64_t strips_len, trace_len;
};

// Batched launch: `grid` CTAs (all resident) of `threads` threads, E points
// per thread (4, 8 or 16).
int launch_batched(const BatchRun& a, int dtype, int E, int threads, int grid, cudaStream_t st);
int max_resident_batched(int dtype, int E, int threads);
// The FP32 instances (compiled in their own translation unit).
int launch_batched_f32(const BatchRun& a, int E, int threads, int grid, cudaStream_t st);
int max_resident_batched_f32(int E, int threads);

// ------------------------------------------------------------ adjoint

// nrods rods of the same N and K, packed rod-major.
struct AdjointRun {
  int64_t nrods, N, K;
  const double* r;         // host, nrods
  const double* c1;        // host, nrods
  const double* cN;        // host, nrods
  int S, q;                // segments per rod and delay window (used when trace != null)
  const uint8_t* trace;    // device [rod][K][S-1][2], null: synchronous run
  const void* u0;          // device, nrods*N values of the dtype
  const double* u_obs;     // device, nrods*N
  int64_t ckpt_every;      // C
  void* uK;                // device, nrods*N values of the dtype, or null
  double* grad_u0;         // device, nrods*N
  double* grad_r;          // host, nrods (may be null)
  double* loss;            // host, nrods (may be null)
  int cotangent;           // 1: u_obs holds dL/du(K) itself (general vector-Jacobian product)
  cudaStream_t stream;
};
// Runs the forward pass with checkpoints and the backward pass; waits for
// the stream.  Returns a heat1d_status.
int run_adjoint(const AdjointRun& a, int dtype);

// Largest number of CTAs of these kernels that can be resident at once.
int max_resident_sync(int dtype, int E, int threads);
int max_resident_async(int dtype, int E, int threads);

}  // namespace heat1d_impl

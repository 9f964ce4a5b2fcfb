/*
 * heat1d.h -- C ABI of libheat1d, a GB300 (sm_103a) solver for the explicit
 * forward-time, central-space (FTCS) update of the 1D heat equation in its
 * synchronous and asynchronous forms.
 *
 * Method: Lee & Bhattacharya, "Asynchronous Parallel Computing Algorithm
 * implemented in 1D Heat Equation with CUDA", arXiv:1510.08982.
 *
 *   Section 2, Eq. (eqn:sync):  u_i(k+1) = r u_{i+1}(k) + (1-2r) u_i(k) + r u_{i-1}(k),
 *                               0 < r <= 1/2, Dirichlet ends u_1 = c1, u_N = c2 (here cN).
 *   Section 3, Eq. (eqn:async): the same update where a neighbour value that
 *                               lives in another processing element (PE) may be
 *                               read from any of the q most recent steps.
 *
 * Conventions shared by every entry point:
 *  - Storage is 0-based and contiguous: u[0] = c1 and u[N-1] = cN are never
 *    updated (and are overwritten with c1, cN when a state is loaded).
 *  - Arithmetic per interior point: v = fma(r, (u[i+1] - 2 u[i]) + u[i-1], u[i]),
 *    the operation order of the paper's printed kernels (Section 4) with one
 *    fused multiply-add.  F64 runs compute in double, F32 runs in float with r,
 *    c1, cN rounded to float.
 *  - The N points are split into S contiguous segments (the PEs of Section 2,
 *    Fig. 1); the first N mod S segments hold one point more.  One CTA owns one
 *    segment.  Asynchrony exists only across segment boundaries (Section 3).
 *  - A delay trace is uint8[K][S-1][2]: entry (k, b, 0) is the delay d with
 *    which segment b read its right neighbour's first point at step k, and
 *    (k, b, 1) the delay with which segment b+1 read its left neighbour's last
 *    point.  The value used was the neighbour's state at step k - d; every
 *    recorded d is < q and <= k.
 *  - Every run is enqueued on the handle's stream and returns at once; its
 *    launch errors are returned directly, its device-side status (a timed-out
 *    wait, a bad trace entry) by heat1d_sync().  Buffers passed in stay owned
 *    by the caller; a pointer flagged on_device must be device memory of the
 *    handle's device.  No C++ exception crosses this boundary.
 *  - Thread safety: a handle must not be used from two host threads at once.
 *    heat1d_last_error() is per host thread.
 */
#ifndef HEAT1D_H
#define HEAT1D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct heat1d* heat1d_t;

enum heat1d_dtype { HEAT1D_F32 = 0, HEAT1D_F64 = 1 };

enum heat1d_status {
  HEAT1D_OK = 0,
  HEAT1D_ERR_INVAL = -1,        /* an argument is out of range */
  HEAT1D_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  HEAT1D_ERR_TIMEOUT = -3,      /* a device-side wait exceeded spin_limit_ns */
  HEAT1D_ERR_NOT_RESIDENT = -4, /* the segments cannot all be resident at once */
  HEAT1D_ERR_TRACE = -5,        /* a replay trace entry is >= q */
  HEAT1D_ERR_OOM = -6,          /* device memory could not be allocated */
  HEAT1D_ERR_BOUNDS = -7        /* bounds-checked build only: a kernel computed an index outside
                                   its buffer; the access was skipped and the run's results are
                                   unspecified */
};

/* Run options.  Zero in a field means "choose automatically". */
typedef struct heat1d_opts {
  int64_t segments;      /* S, the number of segments (PEs).  0: one per SM. */
  int32_t q;             /* delay window of the asynchronous run, 1..255 (Section 3's buffer
                            length q).  0: 3. */
  int32_t halo_steps;    /* T, steps advanced between two exchanges in the synchronous run
                            (overlapped halos of width T) and the block length of the blocked
                            asynchronous run.  0: automatic (on-chip runs: FP64 64, or 32 when the
                            shortest segment has fewer than 4096 points; FP32 512 from 6144 points,
                            256 from 4096, else 128; at most the shortest segment.  Streamed runs 32
                            in FP64, 128 in FP32).
                            1: exchange and grid barrier after every step, as in Section 2. */
  int32_t block_threads; /* threads per CTA for the compute warps (a multiple of 32; at most 512 in
                            streamed runs, which add a loader and a releaser warp).  0: automatic. */
  int32_t elems_per_thread; /* points held in registers per thread (2, 4, 8 or 16, or 32 in F32
                            synchronous and blocked runs; streamed runs 4, 8 or 16).  0: automatic. */
  int64_t spin_limit_ns; /* bound on every device-side wait.  0: 2e9 (2 s). */
  int32_t stall_segment; /* fault injection for tests: when >= 0, that segment of an asynchronous
                            run (that tile of a streamed run; that rod part, by its index among
                            the batch's parts, of a batched run) never publishes, so its
                            neighbours' waits run out and the run ends with HEAT1D_ERR_TIMEOUT.
                            Default -1 (off). */
  int32_t sync_mode;     /* synchronous run: 0 automatic, 1 on-chip (one CTA per segment, the
                            segment in registers), 2 streamed (temporal blocking through HBM:
                            tiles of block_threads * elems_per_thread points, halo_steps steps
                            per pass, each tile copied into shared memory by one bulk copy).
                            Automatic picks on-chip when every segment fits one CTA. */
  int32_t boundary;      /* 0: Dirichlet ends (Section 2).  1: periodic (Section 5.3): the two end
                            points are updated too, each with the other as its outer neighbour;
                            c1 and cN are then unused.  Periodic runs are on-chip synchronous runs
                            and asynchronous runs with S >= 2 (the ring has S boundaries, so a
                            periodic trace is uint8[K][S][2]). */
  int32_t cluster;       /* on-chip asynchronous runs (per-step and blocked): CTAs per thread-block
                            cluster.  Consecutive segments in one cluster hand their edge values
                            (per-step run) or edge strips (blocked run) to each other through
                            distributed shared memory, written straight into the neighbour CTA's
                            shared memory; segments in different clusters exchange through the
                            rings in global memory.  The results and the delay model are the
                            same.  0: automatic (the largest of 8, 4 and 2 that divides S and
                            keeps all S CTAs resident, else 1; blocked runs also need the
                            neighbours' strip rings, 2*R*T values, within 96 KB).  1: no
                            clusters.  2, 4 or 8: that size (HEAT1D_ERR_INVAL if it does not
                            divide S, HEAT1D_ERR_NOT_RESIDENT if it cannot be met). */
  int32_t reserved[4];
} heat1d_opts;

/* Fills *o with the defaults (every field 0 except stall_segment = -1). */
void heat1d_default_opts(heat1d_opts* o);

/* Creates a handle for one rod of N points on the current CUDA device.
 * Requires N >= 3, 0 < r <= 0.5 (Section 2's stability range) and
 * dtype in {HEAT1D_F32, HEAT1D_F64}.  The state starts at zero with the ends
 * set to c1 and cN.  Returns NULL on error (see heat1d_last_error). */
heat1d_t heat1d_create(int64_t N, double r, double c1, double cN, int dtype);

/* Frees the handle and its device memory.  NULL is accepted. */
void heat1d_destroy(heat1d_t h);

/* Message of the last error on this host thread ("" if none). */
const char* heat1d_last_error(void);

/* Sets the CUDA stream (a cudaStream_t; NULL is the legacy default stream). */
int heat1d_set_stream(heat1d_t h, void* stream);

/* Records snapshots of the state during the next runs (the paper keeps the
 * whole history in its array v, Section 4; here it is optional and strided):
 * row j of buf (device, rows x N values of the handle's dtype) receives the
 * state at step j*every of each run, row 0 the state the run starts from.
 * A run of K steps needs K/every + 1 <= rows (else HEAT1D_ERR_INVAL).
 * Synchronous runs need every to be a multiple of the halo depth and must be
 * on-chip.  buf = NULL stops recording.  The buffer stays owned by the
 * caller. */
int heat1d_set_snapshots(heat1d_t h, void* buf, int64_t every, int64_t rows);

/* Replaces the options.  Validates them against N; the segment split and the
 * scratch buffers are rebuilt.  HEAT1D_ERR_INVAL if out of range. */
int heat1d_set_opts(heat1d_t h, const heat1d_opts* o);
int heat1d_get_opts(heat1d_t h, heat1d_opts* o);

/* Number of segments S and, if offsets != NULL, the S+1 segment offsets
 * (host array written by the call). */
int64_t heat1d_num_segments(heat1d_t h, int64_t* offsets);

/* Copies N values (dtype of the handle) into the state; u[0] and u[N-1] are
 * then overwritten with c1 and cN.  on_device: 1 if u is device memory,
 * 0 if host memory (then the call waits for the copy). */
int heat1d_set_u(heat1d_t h, const void* u, int on_device);

/* Copies the current state (N values) out.  With on_device = 0 the call waits
 * for the stream. */
int heat1d_get_u(heat1d_t h, void* u, int on_device);

/* Synchronous run, Section 2 Eq. (eqn:sync): advances the state by K steps.
 * One persistent cooperative launch.  On-chip mode: one CTA per segment holds
 * its segment and T-wide halos in registers, exchanges the halos through
 * global memory and meets the other CTAs at a grid-wide barrier every T steps.
 * Streamed mode (rods too long for on-chip): tiles with T-wide halos are read
 * from HBM, advanced T steps in registers and written back, one pass per T
 * steps, with per-tile pass counters instead of a grid barrier.  Either way
 * the result is identical, bit for bit, to K single steps with a barrier
 * after each. */
int heat1d_run_sync(heat1d_t h, int64_t K);

/* Asynchronous run, Section 3 Eq. (eqn:async): advances the state by K steps
 * with no barrier.  Each segment hands its two edge values on after every
 * step, each value tagged with its version (into the neighbour's shared
 * memory inside a thread-block cluster, else through a ring in global
 * memory), and reads its neighbours' newest version v <= k (waiting only
 * while none >= k-q+1 has arrived).  trace_out (may be
 * NULL) receives the delays actually used, heat1d_trace_bytes(h, K) bytes in
 * the layout above; trace_on_device says where it lives.  Host traces are
 * complete when heat1d_sync() returns. */
int heat1d_run_async(heat1d_t h, int64_t K, uint8_t* trace_out, int trace_on_device);

/* Size in bytes of a trace of K steps: K * (S-1) * 2 (K * S * 2 when periodic). */
int64_t heat1d_trace_bytes(heat1d_t h, int64_t K);

/* Replay of an asynchronous run, Section 3 Eq. (eqn:async) with the delays
 * given: at step k a segment waits for, and uses, exactly the neighbour
 * version k - min(d, k).  Same kernel as heat1d_run_async.  Entries >= q make
 * the run return HEAT1D_ERR_TRACE from heat1d_sync() and leave the state
 * unspecified. */
int heat1d_replay(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device);

/* ------------------------------------------------------------ checkpoint / resume
 *
 * The asynchronous run of Section 3 is the switched system on the augmented
 * state z(k) = [u(k); u(k-1); ...; u(k-q+1)] (Eq. (eqn:async): a read may
 * return any of the q most recent steps).  Only values that cross a segment
 * boundary can be read late, so the augmented state a run needs to continue
 * is u(k) plus every segment's first and last point at the last q steps.
 * After heat1d_run_async or heat1d_replay the handle holds that state; a
 * following asynchronous run or replay continues from it (its step 0 is the
 * global step k, delays are clamped to the global step, its trace covers
 * steps k .. k+K-1), so a run split into several calls equals the run made
 * by one call bit for bit.  Any other state change (heat1d_set_u, a
 * synchronous, blocked or adjoint run, new options) starts over at step 0.
 *
 * State layout: a heat1d_state_header, then N values of u (the handle's
 * dtype), then the history [S][2][q] values: [s][0][j] is segment s's first
 * point and [s][1][j] its last point at global step k-q+1+j.  A state
 * without history (has_history = 0, step 0) holds the current edge values in
 * every history entry. */
typedef struct heat1d_state_header {
  int64_t magic;       /* identifies a heat1d state */
  int64_t step;        /* global step k of the state */
  int64_t N, S;        /* points and segments of the handle that wrote it */
  int32_t q, dtype;    /* delay window and HEAT1D_F32 / HEAT1D_F64 */
  int32_t has_history; /* 1: continues an asynchronous run */
  int32_t reserved;
} heat1d_state_header;

/* Size in bytes of a state: sizeof(heat1d_state_header) + (N + 2*S*q) values. */
int64_t heat1d_state_bytes(heat1d_t h);

/* Copies the handle's state (layout above) into `state` (device or host per
 * on_device, heat1d_state_bytes(h) bytes, owned by the caller); with a host
 * buffer the call waits for the stream. */
int heat1d_get_state(heat1d_t h, void* state, int on_device);

/* Loads a state written by heat1d_get_state of a handle with the same N,
 * segments, q and dtype (else HEAT1D_ERR_INVAL, nothing changed); the next
 * asynchronous run or replay continues it. */
int heat1d_set_state(heat1d_t h, const void* state, int on_device);

/* ------------------------------------------------------------ asynchronous run, temporally blocked
 *
 * The bounded-delay model of Section 3 (Eq. (eqn:async)) applied to blocks of
 * T steps instead of single steps; the paper has no such run (its PEs exchange
 * one value per step), so the model is defined here.  T is the handle's halo
 * depth (heat1d_opts.halo_steps, with the on-chip defaults given there, at
 * most the shortest segment; heat1d_get_opts reports the value in use).  Time is cut into blocks of T
 * steps; in block b (steps bT .. bT+tb-1, tb = min(T, K-bT)) every segment
 * advances tb steps on its own points at step bT plus two T-wide halo strips:
 * its left neighbour's last T points at step (b-dL)T and its right
 * neighbour's first T points at step (b-dR)T, d < q, d <= b.  Its own points
 * after the block are its part of the state at step bT+tb.  With every delay 0
 * this is heat1d_run_sync bit for bit; with T = 1 it is Eq. (eqn:async).
 *
 * Trace layout: uint8 trace[b][boundary][side], ceil(K/T) blocks, S-1
 * boundaries (S on the periodic ring, boundary b joining segments b and
 * (b+1) mod S), the sides as in heat1d_run_async (side 0: segment b's read of
 * its right neighbour; side 1: segment b+1's read of its left neighbour).
 * Periodic runs (boundary = 1) need S >= 2; with S = 2 both halos come from
 * the one neighbour, each strip its own copy. */

/* Rods too long for on-chip segments (sync_mode 2, or sync_mode 0 when a
 * segment does not fit one CTA) run the same model streamed through HBM: the
 * tiles of the streamed synchronous run are the segments (tile j holds points
 * [jW, min((j+1)W, N)); only the last tile may be shorter than T), each block
 * of T = the streamed halo depth steps reads a tile's own points from the
 * state, advances them in registers and writes them back in place, and the
 * tiles' edge strips travel through version rings in HBM.  Such runs need
 * Dirichlet ends (boundary 0).  heat1d_blocked_segments() gives the split
 * and the block length a trace refers to. */

/* Free-running blocked run of K steps: each segment publishes its two edge
 * strips once per block and starts the next block with its neighbours'
 * newest strips not newer than that block, waiting only while one is more
 * than q-1 blocks old.  trace_out (may be NULL; device or host per
 * trace_on_device) receives heat1d_blocked_trace_bytes(h, K) bytes of delays. */
int heat1d_run_async_blocked(heat1d_t h, int64_t K, uint8_t* trace_out, int trace_on_device);

/* Replay of a blocked run with the strip delays given (entries >= q: the run
 * returns HEAT1D_ERR_TRACE from heat1d_sync() and the state is unspecified). */
int heat1d_replay_blocked(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device);

/* Size in bytes of a blocked trace of K steps: ceil(K/T) * (S-1) * 2
 * (ceil(K/T) * S * 2 on the periodic ring), S and T as heat1d_blocked_segments
 * reports them. */
int64_t heat1d_blocked_trace_bytes(heat1d_t h, int64_t K);

/* The segments of the blocked asynchronous run: returns their number S (the
 * handle's segments on chip, the tiles when streamed) and, if offsets is not
 * NULL, writes the S+1 offsets (host array, segment s = [offsets[s],
 * offsets[s+1])); *block_steps (may be NULL) receives T, the steps per block.
 * Negative on a NULL handle. */
int64_t heat1d_blocked_segments(heat1d_t h, int64_t* offsets, int32_t* block_steps);

/* The thread-block cluster size (CTAs per cluster, 1 = none) that the
 * handle's per-step asynchronous runs (blocked = 0: heat1d_run_async,
 * heat1d_replay) or blocked asynchronous runs (blocked = 1:
 * heat1d_run_async_blocked, heat1d_replay_blocked; 1 when streamed) use with
 * its current options (heat1d_opts.cluster).  Negative status on error:
 * HEAT1D_ERR_INVAL for segments too long for the on-chip kernel,
 * HEAT1D_ERR_NOT_RESIDENT when the requested size cannot be met. */
int heat1d_async_cluster(heat1d_t h, int blocked);

/* Bounds-checked build.  The library can be compiled with HEAT1D_CHECKED
 * defined (libheat1d_checked.so): in the on-chip synchronous, per-step
 * asynchronous and blocked kernels, the streamed asynchronous kernel and the
 * batched kernel, every global-memory index computed for the state,
 * snapshots, traces, edge buffers, rings, strips and edge histories (and the
 * range of every bulk copy) is then compared with its buffer's extent before
 * the access; an index outside it skips the access and records
 * HEAT1D_ERR_BOUNDS in the device status word (reported by heat1d_sync /
 * heat1d_batch_sync), without trapping.  Results are otherwise identical.
 * heat1d_checked() returns 1 in that build, 0 in the normal one. */
int heat1d_checked(void);

/* Checked build only: runs one kernel on the current device that computes
 * an index one past the end of a 4-element device buffer for a load and a
 * store; the checks skip both.  Returns HEAT1D_ERR_BOUNDS when they fired
 * (the expected result), HEAT1D_OK if they did not, HEAT1D_ERR_CUDA on a CUDA
 * error.  The normal build returns HEAT1D_ERR_INVAL and launches nothing. */
int heat1d_checked_selftest(void);

/* Waits for the handle's stream and returns the device-side status of the
 * runs enqueued since the previous heat1d_sync(): HEAT1D_OK,
 * HEAT1D_ERR_TIMEOUT or HEAT1D_ERR_TRACE (HEAT1D_ERR_CUDA on a CUDA error). */
int heat1d_sync(heat1d_t h);

/* ------------------------------------------------------------ batched rods
 *
 * Many independent rods of uneven N, r and K advanced by the synchronous
 * update (Section 2, Eq. (eqn:sync)) in one persistent launch.  Rod j lives in
 * u_packed[offset .. offset+N-1] (dtype of the batch; rods must not overlap)
 * and is advanced K steps in place; when K > 0 its ends become c1 and cN.
 * The result for each rod is identical, bit for bit, to heat1d_run_sync on
 * that rod alone. */
typedef struct heat1d_rod {
  int64_t offset; /* first point of the rod in the packed state */
  int64_t N;      /* points, >= 3 */
  int64_t K;      /* steps, >= 0 */
  double r;       /* 0 < r <= 0.5 */
  double c1, cN;  /* Dirichlet ends */
} heat1d_rod;

typedef struct heat1d_batch* heat1d_batch_t;

/* Plans a batch once: validates the rods, sorts the work (warp batches for
 * rods of at most 32 * elems_per_thread points, one CTA for rods that fit a
 * CTA, parts with halo_steps-deep halos for longer rods), uploads the plan
 * and allocates its scratch.  Options used: elems_per_thread (4, 8, 16;
 * default 16 in F32, 8 in F64), block_threads (default 256), halo_steps
 * (default 32 in F32, 16 in F64), spin_limit_ns.  NULL on error. */
heat1d_batch_t heat1d_batch_create(const heat1d_rod* rods, int64_t nrods, int dtype, const heat1d_opts* o);

/* Enqueues one run of the planned batch on `stream` (device pointer
 * u_packed).  Only memsets and one kernel launch: no allocation and no
 * synchronisation, so the call can be captured in a CUDA graph. */
int heat1d_batch_run(heat1d_batch_t b, void* u_packed, void* stream);

/* Asynchronous batched run (the config-4 stretch of Section 3's model): the
 * parts of every rod that is split over several CTAs are the segments of the
 * blocked asynchronous model (Eq. (eqn:async) per block of T = halo_steps
 * steps): after each block a part publishes its first and last T points as a
 * strip version and starts the next block with its neighbouring parts'
 * newest strips not newer than that block, waiting only while one is more
 * than q-1 blocks old (q from heat1d_opts.q at heat1d_batch_create, default
 * 3).  Rods that fit one CTA or one warp have no inner boundary and advance
 * as in heat1d_batch_run.  trace_out (device, heat1d_batch_trace_bytes(b)
 * bytes, or NULL) receives the delays: part by part (see
 * heat1d_batch_rod_parts), uint8[ceil(K/T)][2] per part, [j][0] the delay of
 * its read of the left neighbour in block j, [j][1] of the right one (0 in
 * block 0 and at a rod end).  The launch is capturable in a CUDA graph. */
int heat1d_batch_run_async(heat1d_batch_t b, void* u_packed, void* stream, uint8_t* trace_out);

/* Replay of an asynchronous batched run with the delays given (device, the
 * layout above); an entry >= q makes heat1d_batch_sync return
 * HEAT1D_ERR_TRACE. */
int heat1d_batch_replay(heat1d_batch_t b, void* u_packed, void* stream, const uint8_t* trace);

/* Bytes of the trace of an asynchronous batched run. */
int64_t heat1d_batch_trace_bytes(heat1d_batch_t b);

/* The parts of rod `rod` (its index in the array given to
 * heat1d_batch_create): returns their number P (1 for a rod that is not
 * split); offsets (may be NULL; P+1 entries) receives the parts' first points
 * relative to the rod's start and the rod length last; *trace_offset (may be
 * NULL) the byte offset of its first part's trace (-1 if not split; part p's
 * trace follows at trace_offset + 2*p*ceil(K/T)). */
int64_t heat1d_batch_rod_parts(heat1d_batch_t b, int64_t rod, int64_t* offsets, int64_t* trace_offset);

/* Waits for the last run's stream; returns its device status. */
int heat1d_batch_sync(heat1d_batch_t b);

/* info[8]: warp batches, single-CTA rods, rod parts, CTAs, threads per CTA,
 * elems_per_thread, halo_steps, points per CTA. */
int heat1d_batch_describe(heat1d_batch_t b, int64_t* info);

void heat1d_batch_destroy(heat1d_batch_t b);

/* One-shot form: plan, run, wait, free.  u_packed is a device pointer. */
int heat1d_run_batched(const heat1d_rod* rods, int64_t nrods, void* u_packed, int dtype, const heat1d_opts* o,
                       void* stream);

/* ------------------------------------------------------------ adjoint
 *
 * Gradient of the terminal misfit L = 0.5 * sum_i (u_i(K) - u_obs_i)^2 with
 * respect to u(0) and r.  The paper does not differentiate its scheme; the
 * adjoint here is derived from Section 3, Eq. (eqn:async) (Section 2's
 * Eq. (eqn:sync) when trace is NULL): lambda(K) = u(K) - u_obs on the
 * interior, then backwards lambda_i(k) += (1-2r) lambda_i(k+1) and
 * lambda_{i+-1}(k - d) += r lambda_i(k+1) for every read u_{i+-1}(k - d) the
 * forward step made, and dL/dr = sum_k sum_i lambda_i(k+1) *
 * ((u_{i+1}(k-dR) - 2 u_i(k)) + u_{i-1}(k-dL)).  The gradient at the two
 * Dirichlet entries of u(0) is 0.
 *
 * The forward pass keeps a checkpoint every ckpt_every steps (0: 128): the
 * state plus the last q values of every point next to a segment boundary.
 * The backward pass recomputes each interval from its checkpoint and marches
 * lambda back through it.  lambda has the handle's dtype; the loss and dL/dr
 * are accumulated in FP64 (an FP32 run sums the products of a warp's points
 * in FP32 first) and every reduction is deterministic, the same for any
 * ckpt_every.  grad_u0 is always FP64.  Scratch
 * (checkpoints, one interval of states) is allocated per call and freed;
 * HEAT1D_ERR_OOM if it does not fit.  The call waits for the stream.
 */

/* On the handle: u(0) is the current state; afterwards the state is u(K).
 * trace: NULL for the synchronous run, else the replayed asynchronous run's
 * delays (layout above; host or device per trace_on_device; every entry must
 * be < q, else HEAT1D_ERR_TRACE).  u_obs and grad_u0 are device arrays of N
 * doubles; grad_r and loss are host doubles (may be NULL). */
int heat1d_adjoint(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device, const double* u_obs,
                   int64_t ckpt_every, double* grad_u0, double* grad_r, double* loss);

/* Vector-Jacobian product of the same map u(0), r -> u(K): grad_uK (device,
 * N doubles) is dL/du(K) for any L; returns dL/du(0) and dL/dr. */
int heat1d_vjp(heat1d_t h, int64_t K, const uint8_t* trace, int trace_on_device, const double* grad_uK,
               int64_t ckpt_every, double* grad_u0, double* grad_r);

/* The same for nrods rods of equal N and K packed rod-major in device arrays
 * (u0 and uK of `dtype`, u_obs and grad_u0 of doubles, nrods*N values each;
 * uK may be NULL).  r, c1, cN, grad_r and loss are host arrays of nrods.
 * cotangent = 1 makes u_obs the cotangent dL/du(K) (loss then 0).  trace
 * (device, [rod][K][S-1][2], or NULL) with S = segments and q. */
int heat1d_adjoint_batched(int64_t nrods, int64_t N, int64_t K, const double* r, const double* c1, const double* cN,
                           int dtype, const void* u0, const double* u_obs, int cotangent, int64_t segments, int q,
                           const uint8_t* trace, int64_t ckpt_every, void* uK, double* grad_u0, double* grad_r,
                           double* loss, void* stream);

/* Synchronous run that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- for example
 * code running inside a host callback or an allocator hook, a plug-in that may
 * not grow the process's device memory, or a loop that forbids allocation
 * after start-up.  The handle API allocates state and scratch at
 * heat1d_create(), which such callers cannot do.
 *
 * Computes the same K steps as heat1d_run_sync() with the handle's default
 * options (same kernel and launch-shape rule, same result bit for bit; the
 * halo depth is capped at what its scratch array holds) from u_in to u_out:
 * two distinct device buffers of N values of
 * `dtype`, owned by the caller.  u_out[0] and u_out[N-1] receive c1 and cN.
 * segments: S, in [1, 256], or 0 for one per SM (at most 256); each segment
 * must fit one CTA (about 8K points in F32 and in F64).  The halo depth is
 * F32 128 steps; F64 64 on segments of 4096 points or more, else 32; at most
 * N/S.  The run is enqueued on `stream` (a
 * cudaStream_t, NULL for the legacy default stream).  If status_out is not
 * NULL it must be a device int; it receives the run's device status
 * (HEAT1D_OK or HEAT1D_ERR_TIMEOUT) when the run completes on the stream.
 *
 * The kernel's scratch (halo buffers, barrier counter, status word, segment
 * offsets; about 530 KB) lives in one fixed __device__ array inside the
 * library: every GPU that loads the library holds it until the process exits.
 * Calls reuse it: each call clears what must start at zero, so results never
 * depend on an earlier call, but two calls that overlap on the GPU (different
 * streams, or different host threads, without ordering between them) race on
 * that array and give wrong results.  The call makes the current device's
 * primary context current (cudaSetDevice) unless another context already is.
 * The first call in each CUDA context looks up the array's device address
 * there (cudaGetSymbolAddress) and caches it under the context's id; an
 * address is only valid in its own context, so a device reset, which
 * destroys the context, makes the next call look it up again.  Make that
 * first call on each device before any stream capture begins.  No call
 * allocates device or pinned memory.  Returns HEAT1D_ERR_INVAL (message in
 * heat1d_last_error()) for sizes beyond these limits, HEAT1D_ERR_NOT_RESIDENT
 * if the segments cannot all be resident, HEAT1D_ERR_CUDA when a CUDA call or
 * the launch fails. */
int heat1d_run_sync_noalloc(const void* u_in, void* u_out, int64_t N, double r, double c1, double cN, int dtype,
                            int64_t K, int64_t segments, void* stream, int* status_out);

/* ------------------------------------------------------------ roofline probe
 *
 * Throughput probe of the fused multiply-add pipe that bounds the on-chip runs
 * (the paper has no counterpart: it measures the arithmetic roofline the FTCS
 * kernels are held against, three FP64 fused multiply-adds per update in F64
 * runs).  Enqueues one launch of `blocks` CTAs of `threads` threads (a
 * multiple of 32, at most 1024) on `stream`; every thread advances `chains`
 * (4, 8 or 16) independent chains a <- fma(a, b, c) for `iters` iterations,
 * or, with chains = -P (P = 8 or 16), P points on a ring in registers by two
 * FTCS steps per iteration (three fused multiply-adds per point and step, the
 * stencil kernels' own operand pattern), and writes one value to out
 * (device, blocks * threads values of the dtype, owned by the caller).  *fma_per_launch (may be NULL) receives the number of
 * fused multiply-adds the launch executes; the caller times the launch (CUDA
 * events on the stream) and divides.  HEAT1D_ERR_INVAL for a bad shape, chain
 * count or dtype, HEAT1D_ERR_CUDA if the launch fails. */
int heat1d_probe_fma(int dtype, int chains, int64_t iters, int64_t blocks, int threads, void* out, void* stream,
                     int64_t* fma_per_launch);

#ifdef __cplusplus
}
#endif

#endif /* HEAT1D_H */

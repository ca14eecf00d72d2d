/*
 * sosfilt.h - C ABI of the GB300 (sm_103a) cascaded-biquad filter library.
 *
 * The library filters FP32 signals through a cascade of K second-order
 * sections (biquads), paper Sec. II, Eq. general_cascaded_equation and
 * Eq. complex_second_order:
 *
 *   y_k[n] = b0 x_k[n] + b1 x_k[n-1] + b2 x_k[n-2] - a1 y_k[n-1] - a2 y_k[n-2],
 *   x_1 = x,  x_{k+1} = y_k,  y = y_K,
 *
 * every row first divided by its a0.  The result is the exact solution of the
 * banded block-Toeplitz system of Sec. III, Eq. recursive_equation_block_form
 * (up to FP32 rounding); it is computed with the stride-N multi-block
 * formulation of Sec. V (lane l of a 32-lane warp owns the contiguous samples
 * [lN, lN+N) of a group, i.e. register m of all lanes is the strided block
 * x_m = [x[m], x[m+N], ...]), the PH factorisation of Sec. VI-B for the
 * recursive stage, and one permutation / de-permutation pair per cascade
 * (Sec. VII-B).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named "device" must point to device memory of the current CUDA
 *   device.  The caller owns every buffer; the library never allocates device
 *   memory and never frees anything.
 * - Streams are passed as `void *` holding a cudaStream_t (NULL = the legacy
 *   default stream).  All device work is enqueued on that stream and the call
 *   returns without synchronising; nothing inside calls cudaMalloc or
 *   synchronises the host, so calls may be captured into a CUDA graph.
 * - Channels are packed: channel c occupies samples [off_c, off_c + len_c) of
 *   x and y, off_c being the exclusive prefix sum of the lengths.  Any offset
 *   alignment is accepted (16-byte-aligned channels take a faster load path).
 * - sos rows are FP64 (b0, b1, b2, a0, a1, a2), shape [n_channels][kmax][6];
 *   rows k >= K[c] are not read.  a0 must be nonzero.
 * - State (zi, zf) is FP32 [n_channels][kmax][2] in the transposed direct
 *   form II convention of scipy.signal.sosfilt: for section k,
 *     z1 = b1 x[-1] + b2 x[-2] - a1 y[-1] - a2 y[-2],  z2 = b2 x[-1] - a2 y[-1],
 *   which are exactly the two scalar corrections the paper adds to the first
 *   element of the first two blocks (Sec. V-A, Eq. feedforward_block_uniform).
 *   zf rows k >= K[c] are written as zero; a zero-length channel returns zi.
 * - Errors in arguments are detected on the host and returned before any
 *   work is enqueued.  Errors found on the device (nonzero a0 violated,
 *   non-finite coefficients, an unstable section when the stability check is
 *   on, a look-back wait that ran out) are written to a status word inside
 *   the workspace; read it with sos_device_status().
 */
#ifndef SOSFILT_H
#define SOSFILT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sos_status {
    SOS_OK = 0,
    SOS_ERR_ARG = -1,         /* bad argument (null pointer, size, kmax > 8, ...) */
    SOS_ERR_UNSTABLE = -2,    /* a section has a pole on/outside the unit circle (check on) */
    SOS_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    SOS_ERR_TIMEOUT = -4,     /* a cross-tile look-back wait exceeded its bound */
    SOS_ERR_WORKSPACE = -5,   /* workspace too small or not initialised */
    SOS_ERR_UNSUPPORTED = -6, /* tuning values outside the compiled set */
    SOS_ERR_COEF = -7         /* a0 == 0 or a non-finite coefficient */
} sos_status;

/* Tuning knobs.  Pass NULL for the library defaults.
 *   n_blocks: N, samples per lane per group (the paper's number of blocks):
 *             16, 32 or 64 (0 = default 32).
 *   warps:    W, warps per tile (one tile = W*32*N samples): 4, 8 or 16
 *             (0 = default 8).
 *   algo:     recursive-stage solver: 0 = default (PH), 1 = PH (Sec. VI-B),
 *             2 = cyclic reduction (Sec. VI-C) for every section whose
 *             reduction is well conditioned (max |f_i / e_i| <= 100 over the
 *             log2 N levels; the others keep PH).  CR applies to channels
 *             within their memory horizon (the warp-segment kernel takes CR
 *             for a channel only when all its sections qualify, the section
 *             pipeline section by section); channels carried by the look-back
 *             use PH.
 *   flags:    bit 0 (SOS_FLAG_CHECK_STABLE): reject sections whose poles are
 *             not strictly inside the unit circle.
 *             bit 1 (SOS_FLAG_CARRY_ONLY): carry every channel's state between
 *             tiles by the decoupled look-back, even where the channel's
 *             memory horizon would let its tiles overlap and start from zero
 *             state (same results to rounding; for testing and tuning).
 *             bit 2 (SOS_FLAG_SECTION_PIPELINE): run the channels within their
 *             memory horizon by the section pipeline (one warp per section,
 *             groups handed from warp to warp, segments sized per CTA)
 *             instead of the default warp-segment kernel (one warp filters a
 *             whole segment through all K sections, segments sized to give
 *             every resident warp work).  Segment lengths differ, so the same
 *             flags must reach sos_prepare and sos_apply.  Every section runs
 *             in FP32 there: sections flagged as ill-conditioned
 *             (sos_plan_extended) get extended precision only on the
 *             warp-segment kernel.  The backward runs its own adjoint kernel
 *             whatever this bit.
 *             bit 3 (SOS_FLAG_REPLAN): recompute every channel's tables in
 *             sos_prepare even where the plan cache would keep them (see
 *             sos_prepare; same results, for timing the full plan).
 *             bit 4 (SOS_FLAG_DOUBLE_FLOAT): run every channel within its
 *             memory horizon with double-float samples (precision class 3
 *             of sos_plan_extended), whatever the plan's estimate; about ten
 *             times the arithmetic, for results within about 2^-40 of the
 *             exact ones where FP32 would lose digits.
 *             bits 8..11 (SOS_FLAG_WS_CTAS(n)): CTAs per SM of the
 *             warp-segment launch, 1..15 (0 = as many as fit; more than fit
 *             is clamped).  Fewer, longer-running warps suit calls whose
 *             segments fill the GPU about once (one long signal); the most
 *             that fit suit large batches.
 *
 * Cross-tile state.  The plan bounds each channel's impulse-response tail by
 * partial fractions over its poles and finds its memory horizon P: the warm-up
 * after which the state a tile would drop changes the output by less than
 * 2^-30 relative.  The channel is then cut into segments of S samples (the
 * call's segment length, a multiple of 32 N chosen from its total length, or
 * 2 P rounded up to whole groups when that is longer) that each start P
 * samples early from zero state (no cross-segment dependency).  Coincident
 * poles, where partial fractions fail, get a cruder bound over the largest
 * pole radius r (a tail of the form C(n + 2K - 1, 2K - 1) r^n) when the
 * channel is at least eight of the segments it asks for.  Where no horizon is
 * bounded (a pole within 1e-7 of the unit circle, or coincident poles on a
 * shorter channel), the DF2T state of every section is carried by a
 * decoupled look-back composing FP64-accurate affine maps (Sec. V's group
 * hand-off made parallel). */
typedef struct sos_tuning {
    int32_t n_blocks;
    int32_t warps;
    int32_t algo;
    int32_t flags;
} sos_tuning;

#define SOS_FLAG_CHECK_STABLE 1
#define SOS_FLAG_CARRY_ONLY 2
#define SOS_FLAG_SECTION_PIPELINE 4
#define SOS_FLAG_REPLAN 8
#define SOS_FLAG_DOUBLE_FLOAT 16
#define SOS_FLAG_WS_CTAS(n) (((n) & 15) << 8)
#define SOS_MAX_SECTIONS 8

/* Bytes of device workspace needed for a call with these sizes.
 * lengths_host: host array [n_channels] of channel lengths (>= 0).
 * Returns 0 if the arguments are invalid. */
size_t sos_workspace_size(int32_t n_channels, int32_t kmax, const int64_t *lengths_host,
                          const sos_tuning *tuning);

/* Zero-initialise a workspace once, before its first use (stream-ordered
 * memset).  A workspace may be reused by any number of later calls with sizes
 * that fit, but calls sharing a workspace must not overlap on the GPU. */
sos_status sos_workspace_init(void *workspace, size_t ws_bytes, void *stream);

/* Forward cascade filter (the hot path).
 *   x        device FP32 [sum len]            input signals, packed
 *   sos      device FP64 [n_channels][kmax][6]
 *   K        device int32 [n_channels]        sections per channel, 0..kmax
 *   n_channels >= 1, 1 <= kmax <= 8
 *   lengths       device int64 [n_channels]   channel lengths
 *   lengths_host  host   int64 [n_channels]   the same values (used for sizing)
 *   zi       device FP32 [n_channels][kmax][2] or NULL (zero initial state)
 *   y        device FP32 [sum len]            output (must not overlap x)
 *   zf       device FP32 [n_channels][kmax][2] or NULL
 *   workspace / ws_bytes  device buffer of at least sos_workspace_size() bytes,
 *                         initialised once by sos_workspace_init()
 *   tuning   host pointer or NULL
 *   stream   cudaStream_t as void*
 * Returns SOS_OK once the work is enqueued. */
sos_status sos_filter(const float *x, const double *sos, const int32_t *K, int32_t n_channels,
                      int32_t kmax, const int64_t *lengths, const int64_t *lengths_host,
                      const float *zi, float *y, float *zf, void *workspace, size_t ws_bytes,
                      const sos_tuning *tuning, void *stream);

/* The two halves of sos_filter, for callers that filter many signals with
 * the same coefficients, section counts and lengths (or that time the
 * filtering kernel alone).  sos_apply's kernels are launched with
 * programmatic dependent launch: each may become resident before the kernel
 * ahead of it in the stream has finished, and waits on the device for that
 * kernel's completion (and its memory writes) before it reads anything, so
 * stream order holds as for ordinary launches.
 *
 * sos_prepare enqueues the plan kernel: the per-channel offsets and tile
 * prefix, and the coefficient tables (normalisation by a0, the split-off
 * gain of Sec. II, Eq. simple_second_order, and the transition-matrix powers,
 * "pre-computed before filtering" as in Sec. VI-B, formed in FP64).  It also
 * clears the workspace's device status word.  Plan cache: the workspace
 * keeps, per channel, the raw sos rows (bit for bit), K and length its tables
 * were built from, and the call-level inputs (tuning, kmax, channel count);
 * a channel whose inputs all match keeps its tables and the plan kernel skips
 * it on the device (no host synchronisation), and when every channel matches
 * the dispatch order is kept too.  Changing any coefficient, K, length or
 * tuning recomputes what depends on it.  SOS_FLAG_REPLAN turns the cache off
 * for a call.  sos_plan_recomputed() reports what the latest plan did.
 *
 * sos_apply enqueues only the filtering kernel, reusing those tables; it may
 * be called any number of times after one sos_prepare on the same workspace
 * with the same K, lengths and tuning (x, y, zi and zf may change between
 * calls).  Arguments mean what they mean in sos_filter.
 *
 * sos_filter == sos_prepare followed by sos_apply. */
sos_status sos_prepare(const double *sos, const int32_t *K, int32_t n_channels, int32_t kmax,
                       const int64_t *lengths, const int64_t *lengths_host, void *workspace,
                       size_t ws_bytes, const sos_tuning *tuning, void *stream);
sos_status sos_apply(const float *x, int32_t n_channels, int32_t kmax,
                     const int64_t *lengths_host, const float *zi, float *y, float *zf,
                     void *workspace, size_t ws_bytes, const sos_tuning *tuning, void *stream);

/* The two launches of sos_apply, separately: the kernel for channels within
 * their memory horizon (the warp-segment kernel, or the section pipeline
 * under SOS_FLAG_SECTION_PIPELINE) and the look-back kernel (channels whose
 * state is carried between tiles; it also writes the final states of empty
 * channels and of sections past K).  sos_apply = sos_apply_pipeline then
 * sos_apply_carried on the same stream; the two touch disjoint channels, so
 * they may also run on two streams (both after sos_prepare, both before the
 * outputs are read).  Same arguments and errors as sos_apply.  No
 * counterpart in the paper: a scheduling split of the one operation. */
sos_status sos_apply_pipeline(const float *x, int32_t n_channels, int32_t kmax,
                              const int64_t *lengths_host, const float *zi, float *y, float *zf,
                              void *workspace, size_t ws_bytes, const sos_tuning *tuning,
                              void *stream);
sos_status sos_apply_carried(const float *x, int32_t n_channels, int32_t kmax,
                             const int64_t *lengths_host, const float *zi, float *y, float *zf,
                             void *workspace, size_t ws_bytes, const sos_tuning *tuning,
                             void *stream);

/* Low-latency streaming: filters one block of `chunk` new samples of every
 * channel, carrying each channel's state from the previous block, in one
 * kernel launch (no plan launch, no waits between warps).  The paper's
 * real-time scenario: a signal that arrives in blocks, the state handed from
 * block to block exactly as between groups (Sec. V), the
 * transposed-direct-form-II state of Eq. feedforward_block_uniform's
 * corrections.  A channel within its memory horizon has its block cut into
 * segments, one warp each, warmed up over the horizon (the first from zi),
 * so that a long block is not one warp's sequential walk; other channels
 * take one warp per block.  The segments take zi to be the state this
 * filter left after earlier samples of the same signals (whose response is
 * part of the impulse-response tail the horizon bounds).
 *   x, y      device FP32 [n_channels][chunk], channel-major (y must not
 *             overlap x)
 *   zi        device FP32 [n_channels][kmax][2], the state before this block
 *             (NULL = zero state)
 *   zf        device FP32 [n_channels][kmax][2], receives the state after it
 *             (must not overlap zi: alternate two buffers); rows k >= K[c]
 *             are copied from zi
 *   flags     SOS_STREAM_FOREIGN_STATE: zi is some other state (a caller's
 *             initial condition): segments then also start past that
 *             state's own response; 0 otherwise
 *   workspace a workspace on which sos_prepare has run with the channels'
 *             sos and K, lengths all equal to `chunk`, and the same tuning
 *             (the coefficient tables are reused by every block; prepare
 *             again when the coefficients change)
 * Channels with K[c] = 0 copy x to y.  Precision classes (sos_plan_extended)
 * apply as in sos_filter.  Asynchronous on `stream`; argument errors are
 * returned at once.  Consecutive blocks of a stream must be ordered on the
 * GPU (same stream, or events). */
#define SOS_STREAM_FOREIGN_STATE 1u
sos_status sos_stream(const float *x, float *y, const float *zi, float *zf, int32_t n_channels,
                      int32_t kmax, int64_t chunk, uint32_t flags, void *workspace,
                      size_t ws_bytes, const sos_tuning *tuning, void *stream);

/* The whole call from host memory to host memory: sos_filter on a signal in
 * (pinned) host memory, returning the output there.  The packed signal is cut
 * into blocks of at most `block` samples (whole channels grouped up to it; a
 * longer channel in time pieces whose DF2T states are handed from piece to
 * piece on the device, as between groups, Sec. V); for each block the copy in
 * (a library-owned stream), the filter (sos_filter on `stream`) and the copy
 * out (a second library-owned stream) are ordered by events through two
 * device buffers per direction, so that the copies in and out and the
 * filtering overlap.
 *   x_host, y_host  host FP32, packed as in sos_filter; pinned memory for the
 *                   copies to overlap (pageable memory works, serialised)
 *   sos, K, lengths, zi, zf   device arrays as in sos_filter
 *   workspace       device scratch of at least *ws_bytes of
 *                   sos_filter_host_sizes, initialised by sos_workspace_init
 *   staging         device buffer of at least *staging_bytes (the block
 *                   buffers, the state hand-off, two length cells)
 *   block           samples per block (<= 0: an eighth of the signal, at
 *                   least 2^20)
 * Asynchronous on `stream`: y_host holds the output once `stream` has
 * completed the call's work; after an error part way, `stream` still waits
 * for the copies already enqueued, so that the buffers may be released once
 * it is done.  SOS_ERR_WORKSPACE if a buffer is too small;
 * refused (SOS_ERR_ARG) while `stream` is being captured.  Calls on one
 * device enqueue in turn (a library mutex); their copies share the library's
 * two copy streams. */
sos_status sos_filter_host_sizes(int32_t n_channels, int32_t kmax, const int64_t *lengths_host,
                                 int64_t block, const sos_tuning *tuning, size_t *ws_bytes,
                                 size_t *staging_bytes, int64_t *block_used);
sos_status sos_filter_host(const float *x_host, const double *sos, const int32_t *K,
                           int32_t n_channels, int32_t kmax, const int64_t *lengths,
                           const int64_t *lengths_host, const float *zi, float *y_host, float *zf,
                           void *workspace, size_t ws_bytes, void *staging, size_t staging_bytes,
                           int64_t block, const sos_tuning *tuning, void *stream);

/* The comparison algorithms of the paper's evaluation (Sec. VIII, beside
 * PH and cyclic reduction), on the same tables and the same parallel
 * decomposition: each channel cut into segments of seg_len outputs (>= 32),
 * every segment computed from its channel's memory horizon P earlier from
 * zero state (the channel's zi for its first segment; a channel without a
 * horizon is one segment), so that only the filtering of a segment differs.
 *   algorithm 0: scalar -- one thread per segment runs each section's
 *                recursion (Sec. II, Eq. complex_second_order) sample by
 *                sample in FP32;
 *   algorithm 1: block filtering (Sec. IV, Eq. block_filtering_equation) --
 *                one warp per segment, blocks of L = 32 samples (one per
 *                lane), each block and section as H x_n + H_b xbar_{n-1} -
 *                H_a ybar_{n-1} with H the Toeplitz matrix of the section's
 *                first 32 impulse-response samples: 32 + 4 block FMAs per
 *                block.
 * Arguments as in sos_apply (after sos_prepare on the same workspace, same
 * tuning).  Every section runs in FP32 whatever its precision class.  For
 * measurement against the method; not a faster path.  No counterpart
 * beyond the algorithms themselves. */
sos_status sos_apply_baseline(int32_t algorithm, const float *x, int32_t n_channels, int32_t kmax,
                              const int64_t *lengths_host, const float *zi, float *y, float *zf,
                              int64_t seg_len, void *workspace, size_t ws_bytes,
                              const sos_tuning *tuning, void *stream);

/* Zero-phase (forward-backward) filtering: y = R H R H x, H the cascade
 * from zero state and R time reversal within each channel, so that the
 * overall response is |H(e^jw)|^2 with no phase shift (the cascade applied
 * to the signal and again to its time reversal).  No edge padding and no
 * initial-condition matching: the plain composition (callers that want
 * scipy's odd-extension padding pad x themselves).  Arguments as in
 * sos_filter, plus tmp: device FP32 [sum len], caller-owned scratch for the
 * intermediate signal (none of x, y, tmp may overlap).  Five launches on
 * `stream` (plan, forward pass, reversal, forward pass, reversal).  No
 * counterpart in the paper: a use of the paper's filter, the cascade run
 * twice. */
sos_status sos_filtfilt(const float *x, const double *sos, const int32_t *K, int32_t n_channels,
                        int32_t kmax, const int64_t *lengths, const int64_t *lengths_host, float *y,
                        float *tmp, void *workspace, size_t ws_bytes, const sos_tuning *tuning,
                        void *stream);

/* sos_filter without a caller-allocated workspace (the paper has no
 * counterpart; this is a deployment convenience).  Some callers cannot call
 * cudaMalloc at all: real-time audio or control callbacks where its latency
 * and implicit device synchronisation are not allowed, plug-ins running
 * inside a host application that owns the device allocator, and services
 * that must not grow their memory footprint after start-up.  This entry point
 * allocates nothing: its scratch is a fixed 8 MiB array in the library's own
 * device memory (held by every GPU that loads the library until the process
 * exits).  The caller still provides x, sos, K, lengths, zi, y and zf exactly
 * as for sos_filter.
 *   - The first call on a device (with that device current) looks up the
 *     array's device address and zeroes it on `stream`, then waits for
 *     `stream` so that the zeroing has finished before any later call on any
 *     stream; make that first call before any stream capture (during a
 *     capture it returns SOS_ERR_ARG).  It allocates nothing and calls no
 *     allocating routine.
 *   - Sizes whose workspace (sos_workspace_size) exceeds 8 MiB are rejected
 *     with SOS_ERR_WORKSPACE; nothing is enqueued.
 *   - Every call shares the one array and leaves its contents behind; calls
 *     that overlap on the GPU (different streams without ordering, or other
 *     host threads) race with each other and give wrong results.
 *   - device_status: NULL, or a host int32 that receives the device-side
 *     status of this call; passing it makes the call wait for `stream`, so it
 *     must be NULL while `stream` is being captured (else SOS_ERR_ARG).
 * Returns SOS_OK once the work is enqueued (and, with device_status, done). */
sos_status sos_filter_static(const float *x, const double *sos, const int32_t *K,
                             int32_t n_channels, int32_t kmax, const int64_t *lengths,
                             const int64_t *lengths_host, const float *zi, float *y, float *zf,
                             const sos_tuning *tuning, void *stream, int32_t *device_status);

/* Waits for `stream`, then returns (and clears) the device-side status word
 * of the most recent call that used this workspace. */
sos_status sos_device_status(void *workspace, void *stream);

/* Bytes of device workspace for sos_filter_backward with these sizes: the
 * forward workspace, then the forward-state checkpoints of the adjoint
 * kernel (each section's DF2T state at the start of every group of 32 N
 * samples, two slots per group so that neighbouring segments of a channel
 * never share one: 2 * kmax floats per slot) and 5 doubles per (channel,
 * section) for the coefficient sums.  No per-section signal is stored.
 * 0 if invalid. */
size_t sos_backward_workspace_size(int32_t n_channels, int32_t kmax, const int64_t *lengths_host,
                                   const sos_tuning *tuning);

/* Gradients of a loss L through sos_filter (reverse mode, the transpose of
 * the banded-Toeplitz system of Eq. recursive_equation_block_form): given
 * grad_y = dL/dy (device, packed like y) and grad_zf = dL/dzf ([C][kmax][2],
 * may be NULL = zero), writes grad_x = dL/dx (packed like x), grad_sos =
 * dL/d(sos) ([C][kmax][6] float64, w.r.t. the rows as given, a0 included;
 * zero rows past K[c]) and grad_zi = dL/dzi ([C][kmax][2], may be NULL).
 * x, sos, K, lengths, zi are those of the forward call.
 * Per section the adjoint state runs backwards in time with A^T, i.e. the
 * time-reversed all-pole recursion lambda_n = g_n - a1 lambda_{n+1} -
 * a2 lambda_{n+2} started from dL/dzf, then dL/du = b0 lambda_n +
 * b1 lambda_{n+1} + b2 lambda_{n+2}; dL/db_j = sum lambda_{n+j} u_n,
 * dL/da_j = -sum lambda_{n+j} y_n, dL/dzi = (lambda_0, lambda_1).  The
 * section signals are not stored: a forward pass over each segment keeps only
 * the section states at group starts (checkpoints, in the workspace), and the
 * adjoint pass recomputes each group's section inputs from its checkpoint in
 * shared memory just before running that group backwards.
 * Channels are cut into segments warmed up over their memory horizon on both
 * sides; cascades whose poles coincide get a cruder horizon that needs no
 * partial fractions (the largest pole radius r: a tail bound of the form
 * C(n + 2K - 1, 2K - 1) r^n).  Channels with no horizon at all (a pole
 * within 1e-12 of the unit circle) run as one segment each (correct, but
 * without parallelism inside the channel).  Asynchronous on `stream`;
 * argument errors are returned at once, device errors go to the status word. */
sos_status sos_filter_backward(const float *x, const double *sos, const int32_t *K,
                               int32_t n_channels, int32_t kmax, const int64_t *lengths,
                               const int64_t *lengths_host, const float *zi, const float *grad_y,
                               const float *grad_zf, float *grad_x, double *grad_sos,
                               float *grad_zi, void *workspace, size_t ws_bytes,
                               const sos_tuning *tuning, void *stream);

/* Waits for `stream`, then copies from the channel table of the most recent
 * sos_prepare on this workspace, for channels [first, first + count): the
 * memory horizon P of each (>= 0: tiles overlap by P samples and start from
 * zero state; -1: the state is carried by the look-back) into horizon[i] and
 * its tile count into tiles[i] (host arrays of `count` entries; either may be
 * NULL).  Reads the table in fixed pieces: no allocation.  SOS_ERR_ARG if the
 * range is outside the channels of that call.  This query has no counterpart
 * in the paper; it reports how the plan split the work. */
sos_status sos_plan_query(void *workspace, int32_t first, int32_t count, int32_t *horizon,
                          int32_t *tiles, void *stream);

/* Waits for `stream`, then writes for channels [first, first + count) of the
 * most recent sos_prepare on this workspace its precision class into
 * extended[i] (a host array of `count` entries).  The bulk of the method runs
 * in FP32 with FP64-accurate transition powers (Sec. VI-B); where the plan
 * finds that FP32 would lose digits it adds precision, and reports how:
 *   0  every section in FP32;
 *   1  some section's in-lane recursions add the low parts of a1, a2 (FP32
 *      rounding of a1, a2 displaces its poles by more than 2^-18 of their
 *      distance to the unit circle);
 *   2  some section also runs its lane scan and fold (S4) in double-float
 *      (the largest entry of its transition powers A^(N 2^j), A^(N l) exceeds
 *      8, or the displacement exceeds 1e-4);
 *   3  sections run with double-float samples (about 44 bits): the plan's
 *      estimate of the error that FP32 rounding of the signal handed from
 *      section k to k + 1 would cause at the output (white input, from the
 *      norms of the partial cascades by partial fractions) exceeds 2^-15 for
 *      some k, or a section's own rounding (its condition number
 *      ||g|| ||b|| / ||h||) exceeds 2^-17.  The double-float range spans
 *      both sides of every such hand-off and every such section; the
 *      sections outside it run in FP32 (the whole cascade when the estimate
 *      is unreliable or SOS_FLAG_DOUBLE_FLOAT was given).
 * Classes 1..3 take effect on the warp-segment kernel (the default for
 * channels within their memory horizon); the section pipeline
 * (SOS_FLAG_SECTION_PIPELINE), the cyclic-reduction solver and the look-back
 * kernel run every section in FP32.  No allocation.  SOS_ERR_ARG if the
 * range is outside the channels of that call or `extended` is NULL.  This
 * query has no counterpart in the paper. */
sos_status sos_plan_extended(void *workspace, int32_t first, int32_t count, int32_t *extended,
                             void *stream);

/* Sets the bound on every device-side wait of later calls on this workspace
 * (the look-back's polls for a predecessor tile's state, the hand-overs
 * between the warps of one CTA): `limit` polls, or the compiled default for
 * 0 (sos_workspace_init also restores the default).  A wait that runs out
 * records SOS_ERR_TIMEOUT in the workspace's status word and the kernel
 * carries on with what it has (wrong values, but every access stays in
 * bounds and the kernel completes), so that a hung predecessor cannot hang
 * the GPU; a small limit lets a caller test that path.  The copy is ordered
 * on `stream` and waited for, so not for use during a stream capture.  No
 * counterpart in the paper. */
sos_status sos_workspace_set_wait_limit(void *workspace, uint32_t limit, void *stream);

/* Waits for `stream`, then writes into *channels the number of channels
 * whose tables the most recent sos_prepare on this workspace recomputed (0:
 * every channel's tables and the dispatch order came from the plan cache;
 * see sos_prepare).  No allocation.  No counterpart in the paper. */
sos_status sos_plan_recomputed(void *workspace, int32_t *channels, void *stream);

/* Human-readable name of a status code (static string). */
const char *sos_status_str(sos_status status);

/* Library version, for the bindings' sanity check. */
int32_t sos_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SOSFILT_H */

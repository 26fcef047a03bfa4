/*
 * tfft.h -- C ABI of a single-GPU (GB300, sm_103a) transpose-algorithm
 * multidimensional FFT on a virtual Cartesian process grid.
 *
 * The method is that of Dalcin, Mortensen & Keyes, "Fast parallel
 * multidimensional FFT using advanced MPI" (arXiv:1804.09536): a d-D DFT is
 * computed one axis at a time as batched 1-D FFTs (Eq. fftn_forward), and
 * between the partial transforms the array is redistributed so that the next
 * axis is held in full by every process (Eq. general_gt, Eq. gt).  Here the
 * processes are virtual: every "rank" is a block of one device buffer.
 *
 * Conventions used by every call below.
 *
 *  - Global shape N[0..d-1], C row-major (Sec. 3).  1 <= d <= 4.
 *  - Process grid M[0..g-1], 0 <= g <= d-1 (Sec. 3.6); rank p has row-major
 *    coordinates (p_0, ..., p_{g-1}) (Sec. 3.4).  g = 1 is the slab method
 *    (Eqs. slab0-slab1), g = 2 the pencil method (Eqs. pencil0-pencil2).
 *  - Stages s = 0 .. g.  In stage s grid direction i cuts axis i if
 *    i < g - s, else axis i + 1.  Stage 0 is the input alignment; stage g
 *    holds axis 0 in full and is the alignment of the forward output (axes are
 *    not permuted, Sec. 3.3.1 end).  Each cut axis uses the balanced
 *    block-contiguous decomposition of Eq. decompose / Alg. 1.
 *  - Stage buffer: each rank's local array in C order, the ranks' arrays
 *    concatenated in rank order.  tfft_plan_local_box() gives every rank's
 *    block and offset.
 *  - Elements are complex64 (interleaved float re, im; 8 bytes) except the
 *    real stage-0 buffer of a real-to-complex plan (float32).  The complex
 *    global shape of a real-to-complex plan is N[0..d-2], N[d-1]/2 + 1
 *    (footnote to Eq. multifft).
 *  - Sign: TFFT_FORWARD = -1 (exp(-i k x)), TFFT_BACKWARD = +1, as in the
 *    appendix listings.  Normalisation (Eqs. 1-2, Eq. multifft): the forward
 *    transform carries 1/prod(N), the backward none; TFFT_NORM_BACKWARD moves
 *    the factor to the backward transform.  The factor is formed in double
 *    precision and applied once, in the last pass, as a float.
 *
 * Memory ownership: the library never allocates device memory.  Every device
 * buffer (plan state, inputs, outputs, workspace) is allocated and freed by
 * the caller; the plan itself is a host object.  Every device pointer must be
 * 16-byte aligned.  Calls are asynchronous on the given stream (a
 * cudaStream_t passed as void*; NULL is the legacy default stream) and do not
 * synchronise, except the set-up calls tfft_plan_bind(), tfft_batch_bind(),
 * tfft_batch_autotune() and tfft_batch_set_variant(), which return after
 * their copies (and, for the autotuner, its timed runs) are complete.
 *
 * Errors: every call returns a tfft_status.  Arguments are validated before
 * anything is launched; on an error nothing is launched and
 * tfft_last_error() returns a message (per thread).  A CUDA launch error is
 * reported as TFFT_ECUDA; errors of kernels already running surface on a
 * later call or on the caller's synchronisation.  No call traps the device.
 */
#ifndef TFFT_H
#define TFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TFFT_MAX_DIMS 4
#define TFFT_MAX_GRID_DIMS 3

typedef struct tfft_plan_s *tfft_plan;

enum { TFFT_FORWARD = -1, TFFT_BACKWARD = +1 };
enum { TFFT_C2C = 0, TFFT_R2C = 1 };
/* precision: FP32 butterflies everywhere, or the last radix-16 stage on the
   tensor cores with split hi/lo BF16 or FP16 operands (FP16 range-scaled per
   line by a power of two) and FP32 accumulation, in length-512 contiguous
   passes and in the TMA-staged strided passes of lengths 512 and 256 (other
   passes stay FP32) */
enum { TFFT_FP32 = 0, TFFT_TC_BF16X3 = 1, TFFT_TC_FP16X3 = 2 };
/* plan flags */
enum {
  TFFT_NORM_FORWARD = 0,
  TFFT_NORM_BACKWARD = 4,
  TFFT_NO_TMA = 8, /* plain load/store passes even where the TMA-staged ones apply */
  TFFT_NO_GRAPH = 16 /* tfft_execute never replays captured launches (see tfft_execute) */
};
/* execution modes of tfft_execute */
enum {
  TFFT_MODE_FUSED = 0,   /* redistributions fused into the FFT passes' loads/stores */
  TFFT_MODE_UNFUSED = 1, /* FFT passes + one subarray exchange kernel per redistribution */
  TFFT_MODE_PACKED = 2   /* FFT passes + pack (local transpose) -> all-to-all copy -> unpack */
};

typedef enum {
  TFFT_OK = 0,
  TFFT_EINVAL = 1,       /* bad argument (shape, grid, axis, stage, sign, pointer) */
  TFFT_EUNSUPPORTED = 2, /* valid request this build does not implement (e.g. a prime length > 2048) */
  TFFT_EALIGN = 3,       /* a device pointer is not 16-byte aligned */
  TFFT_EWORKSPACE = 4,   /* workspace missing or too small */
  TFFT_ECUDA = 5,        /* a CUDA runtime call failed */
  TFFT_ESTATE = 6        /* plan not bound to a device state buffer */
} tfft_status;

/* Human-readable name of a status code (static string). */
const char *tfft_status_string(int status);
/* Detail of the last error on the calling thread (static per-thread buffer). */
const char *tfft_last_error(void);
/* ABI version, major * 100 + minor. */
int tfft_version(void);

/*
 * Balanced block-contiguous decomposition, Eq. decompose / Alg. 1 (Sec. 3.1):
 * part p of N elements split in M parts has n = q + (r > p) elements starting
 * at s = q p + min(r, p), q = N / M, r = N mod M.  Requires N >= 0, M > 0,
 * 0 <= p < M; n and s must be non-NULL host pointers.
 */
int tfft_decompose(int64_t N, int64_t M, int64_t p, int64_t *n, int64_t *s);

/*
 * Create a plan for a d-D transform of global shape shape[0..ndims-1] on a
 * grid_ndims-D virtual process grid grid[0..grid_ndims-1] (Sec. 3.4; the grid
 * is taken as given, no dims-create balancing).  kind: TFFT_C2C or TFFT_R2C
 * (real input, Hermitian half on the last axis; N[d-1] even).  precision:
 * TFFT_FP32, TFFT_TC_BF16X3 or TFFT_TC_FP16X3.  flags: TFFT_NORM_FORWARD or
 * TFFT_NORM_BACKWARD, optionally | TFFT_NO_TMA | TFFT_NO_GRAPH.
 * Complex lengths that factor into 2, 3 and 5 (<= 4096) run mixed-radix
 * Stockham passes; any other complex length <= 2048 runs Bluestein's
 * convolution form of the DFT (two power-of-two FFTs of length >= 2N - 1 with
 * FP64-built chirp tables) in the same pass structure.  Longer other lengths
 * (and an r2c half-length without a 2/3/5 plan) leave the plan able to
 * redistribute, but its tfft_execute() and tfft_partial() return
 * TFFT_EUNSUPPORTED.
 * The plan is a host object; destroy it with tfft_plan_destroy().
 */
int tfft_plan_create(tfft_plan *plan, int ndims, const int64_t *shape, int grid_ndims,
                     const int *grid, int kind, int precision, int flags);
int tfft_plan_destroy(tfft_plan plan);

/* Number of stages (grid_ndims + 1) and of virtual ranks (product of the grid). */
int tfft_plan_num_stages(tfft_plan plan, int *nstages);
int tfft_plan_num_ranks(tfft_plan plan, int *nranks);
/* Axis newly held in full by a stage: grid_ndims - stage (Sec. 3.3-3.6). */
int tfft_plan_stage_axis(tfft_plan plan, int stage, int *axis);
/* Elements of a whole stage buffer.  real != 0 asks for the real stage-0
   buffer of an R2C plan (stage must be 0). */
int tfft_plan_stage_elems(tfft_plan plan, int stage, int real, int64_t *elems);
/* Block of one rank in a stage: start[d], size[d] (global index space) and the
   element offset of its local array in the stage buffer.  Host pointers. */
int tfft_plan_local_box(tfft_plan plan, int stage, int real, int rank, int64_t *start,
                        int64_t *size, int64_t *offset);

/*
 * Plan state: tables the kernels read (rank offsets, twiddle factors,
 * column blocks, subarray boxes).  The caller allocates tfft_plan_state_bytes()
 * bytes of device memory and passes it to tfft_plan_bind(), which uploads the
 * tables and generates the twiddle factors on the device in double precision
 * (then rounds them to float).  The state must stay allocated and unmodified
 * while the plan is used; bind again after moving it.  Binding records the
 * current device: every later call that launches work on the plan (execute,
 * adjoint, redistribute, partial, the loss calls, host transforms, the
 * device status read) requires that device to be current and otherwise
 * returns TFFT_EINVAL without launching.
 */
int tfft_plan_state_bytes(tfft_plan plan, size_t *bytes);
int tfft_plan_bind(tfft_plan plan, void *d_state, size_t bytes, void *stream);

/*
 * Workspace of tfft_execute() in a mode, in bytes.  TFFT_MODE_FUSED: 0 for
 * C2C (the input buffer is then overwritten) -- pass one stage buffer's worth
 * to keep the input; R2C always needs one complex stage buffer, stored with
 * padded rows when the gathering pass along axis d-2 runs TMA-staged over a
 * column window (odd Hermitian half on a 2-D grid: then slightly more than a
 * stage buffer; always allocate what this call reports).  UNFUSED and
 * PACKED: two complex stage buffers.
 */
int tfft_plan_workspace_bytes(tfft_plan plan, int mode, int keep_input, size_t *bytes);

/*
 * Global redistribution of Alg. 3 / Eq. gt between two adjacent stages:
 * from the stage that holds axis_v in full (input, aligned in v) to the stage
 * that holds axis_w in full (output, aligned in w), within the one-dimensional
 * subgroups of the grid direction that moves.  All subgroups exchange
 * concurrently in one launch; every (sender, receiver) pair copies one
 * subarray box straight from the input to the output (the all-to-all-w of
 * subarray types).  Bit-exact copy.  in and out are stage buffers of the
 * plan's complex shape and must not overlap.
 */
int tfft_redistribute(tfft_plan plan, int axis_v, int axis_w, const void *in, void *out,
                      void *stream);

/*
 * Partial transform F_axis (Sec. 2, the appendix's sequential routine): 1-D
 * DFT of sign `sign` along `axis` of every rank's local array in `stage`, in
 * place.  axis must be held in full in that stage.  The forward direction
 * includes 1/N_axis (Eq. multifft), the backward none.
 */
int tfft_partial(tfft_plan plan, int stage, int axis, int sign, void *inout, void *stream);

/*
 * Whole transform.  sign TFFT_FORWARD: in = stage-0 buffer (float32 for R2C),
 * out = stage-g buffer (Eqs. pencil0-pencil2 and their d-D form).
 * TFFT_BACKWARD: in = stage-g buffer, out = stage-0 buffer (the forward steps
 * reversed, App. A).  mode selects the fused path or one of the two
 * comparison paths; all three give the same result.  work / work_bytes: see
 * tfft_plan_workspace_bytes().  When work is NULL in TFFT_MODE_FUSED C2C the
 * input buffer is used as scratch; a complex-to-real backward always
 * overwrites its input.  in and out must not overlap.
 * Repeated calls: the second call with the same direction, mode, buffers
 * (and, for the adjoint and loss calls, the same coefficient) captures its
 * launches into a CUDA graph on a stream of the plan's own, and that call
 * and every later identical one launch the graph on `stream` instead -- the
 * same kernels with the same arguments, without the per-launch host cost
 * (a few microseconds per kernel).  The plan keeps at most 8 such graphs
 * (least recently used dropped; the cache is locked, so several threads may
 * execute one plan) and destroys them with the plan; launch
 * events (tfft_plan_set_launch_events) and TFFT_NO_GRAPH turn it off, and
 * tfft_execute_host does not use it.  Instantiating a graph (the second
 * identical call) may synchronise the device once.  A
 * caller that frees a buffer and gets the same address back for a new one
 * simply replays the same launches on it.
 */
int tfft_execute(tfft_plan plan, int sign, int mode, const void *in, void *out, void *work,
                 size_t work_bytes, void *stream);

/*
 * Adjoint F^H of the forward transform F of this plan (complex-to-complex
 * plans): stage g -> stage 0.  With the paper's normalisation (1/N on the
 * forward, Eq. multifft) F^H = (1/N) x backward (Eq. 2 is unscaled), so this
 * runs the backward passes -- the forward's passes in reverse order, each
 * redistribution reversed (a permutation, whose adjoint is its inverse) --
 * with 1/N applied in the last pass (no factor under TFFT_NORM_BACKWARD).
 * d_coef (device memory, 8-byte aligned, may be NULL): the result is
 * multiplied by d_coef[0], read on the device by the last pass, so a scalar
 * known only on the GPU (an upstream gradient) costs no extra sweep and no
 * host synchronisation.  Other arguments as tfft_execute().
 */
int tfft_adjoint(tfft_plan plan, int mode, const void *in, void *out, void *work, size_t work_bytes,
                 const double *d_coef, void *stream);

/*
 * Transforms of a sequence of arrays in page-locked host memory, with the
 * copies overlapped: for k = 0 .. count-1, h_in[k] (stage 0 for a first
 * forward, stage g for a first backward; real for an r2c forward) is copied
 * to the GPU, the fused transforms signs[0], signs[1], ... (alternating
 * directions, e.g. {-1, +1} = forward then inverse) run on it, and the result
 * is copied back to h_out[k].  Arrays alternate between two device buffer
 * sets carved from d_space (caller-allocated, device memory, 256-byte
 * aligned, at least tfft_host_space_bytes): the copy-in of array k+1 and the
 * copy-out of array k-1 run on two library-owned streams while array k is
 * transformed on `stream`.  Stream-ordered: the work starts after what was
 * queued on `stream` before the call, and `stream` waits for the last
 * copy-out.  Host pointers that are not page-locked are rejected
 * (TFFT_EINVAL: the copies could not overlap); h_in[k] is not modified.  The
 * first call creates the two streams on the current device; later calls must
 * use the same device.  Not for CUDA graph capture.  The paper has no
 * counterpart (its arrays live in each rank's host memory).
 */
int tfft_host_space_bytes(tfft_plan plan, size_t *bytes);
int tfft_execute_host(tfft_plan plan, int nsigns, const int *signs, int count, const void *const *h_in,
                      void *const *h_out, void *d_space, size_t space_bytes, void *stream);

/*
 * Spectral-weight loss sum_k |y_k w_k|^2 over a whole stage buffer: y is
 * complex64, w is float32 in the same layout (w[i] weighs y[i]); each term and
 * each thread's running sum are carried in compensated FP32 (about 48 bits),
 * the rest in double, in a fixed order (deterministic); the sum is written to
 * d_loss[0] (device memory).  When u is not NULL the same sweep writes
 * u = w^2 y (complex64, same layout; u may alias y): the gradient of
 * g * loss(F x) is then tfft_weighted_energy_grad(u, d_g = &g), i.e.
 * tfft_adjoint(u) with d_coef = 2 g.  Uses scratch
 * inside the plan state: calls on one plan must not overlap on the GPU.
 */
int tfft_weighted_energy(tfft_plan plan, int stage, const void *y, const float *w, double *d_loss,
                         void *u, void *stream);

/*
 * Gradient seed of that loss: z = c * w^2 * y elementwise, c = scale * d_coef[0]
 * (read on the device; d_coef may be NULL for c = scale).  With c = 2 g, the
 * gradient of g * loss(F x) with respect to x is tfft_adjoint(z)
 * (d/dRe x + i d/dIm x convention).  z may alias y.
 */
int tfft_weight_scale(tfft_plan plan, int stage, const void *y, const float *w, const double *d_coef,
                      double scale, void *z, void *stream);

/*
 * Gradient of g * loss(F x) for the loss of tfft_weighted_energy():
 * 2 g F^H(u), u = w^2 F(x) as that call wrote it (stage g), result in stage
 * 0 (d/dRe x + i d/dIm x convention; the chain rule of Sec. 2's linear map
 * F, whose adjoint is tfft_adjoint).  The factor 2 is applied with the
 * adjoint's own 1/N on its last pass, g is read there on the device from
 * d_g (device memory, 8-byte aligned; NULL means g = 1), so the factor costs
 * no sweep and no host synchronisation.  Complex-to-complex plans; other
 * arguments as tfft_adjoint().
 */
int tfft_weighted_energy_grad(tfft_plan plan, int mode, const void *u, void *out, void *work,
                              size_t work_bytes, const double *d_g, void *stream);

/* Number of kernel launches tfft_execute() makes in a mode and direction. */
int tfft_plan_num_launches(tfft_plan plan, int sign, int mode, int *nlaunches);

/*
 * Launch `index` of tfft_execute() in a direction and mode: the kernel's
 * name (NUL-terminated, truncated to name_len) and its algorithmic bytes --
 * one read and one write of every element it moves (complex64), the figure
 * a roofline divides by the launch's duration.  Names: fft_contig_L<n>,
 * fft_strided_L<n> (plain tiles), fft_strided_tma_L<n> (TMA-staged tiles),
 * ..._tma_groups_... (rank groups of an uneven layout), ..._tma_window_...
 * (a column window of a real-to-complex pencil plan; the next launch is the
 * plain kernel over the remaining columns, and each reports the bytes of
 * its own columns), ..._tc_bf16x3 / _tc_fp16x3 (tensor-core stage),
 * fft_strided_bluestein_L<n>, fft_r2c_L<n> / fft_c2r_L<n>, box_copy.
 */
int tfft_plan_launch_info(tfft_plan plan, int sign, int mode, int index, char *name,
                          int name_len, int64_t *bytes);

/*
 * The copy tasks of launch `index` of tfft_execute() in a direction and mode
 * when that launch is a subarray box copy (Alg. 3's exchange, or the pack,
 * all-to-all copy and unpack of TFFT_MODE_PACKED): task t copies nrows rows
 * of rowlen contiguous complex64 elements, row r from in[src + r ss] to
 * out[dst + r ds] (element offsets into the launch's input and output
 * buffers).  Writes min(max_tasks, count) tasks as 6 int64 values each
 * (src, dst, ss, ds, nrows, rowlen) to `tasks` (host memory, may be NULL
 * when max_tasks is 0) and the count to *ntasks.  Host only; TFFT_EINVAL if
 * the launch is not a box copy.  For inspection and tests of the planner.
 */
int tfft_plan_copy_tasks(tfft_plan plan, int sign, int mode, int index, int64_t *tasks, int64_t max_tasks,
                         int64_t *ntasks);

/*
 * Device status word of the plan's state buffer (nothing else writes it):
 * bit 0 (value 1) is set when a kernel gave up on a bounded wait for one of
 * its own asynchronous copies or tensor-core operations (the kernel then
 * stops and its output is incomplete); bit 1 (2) when a TMA tile buffer was
 * not 128-byte aligned (the copy was skipped); bit 2 (4) when, after such a
 * give-up, tensor-core operations were still running at the end of a
 * bounded clean-up wait, so the CTA left its tensor memory allocated rather
 * than release memory still being written.  Synchronises `stream`;
 * reset != 0 clears the word afterwards.
 */
int tfft_plan_device_status(tfft_plan plan, int *status, int reset, void *stream);

/*
 * Polls a TMA pass makes on one of its copy barriers before it gives up
 * (status bit 1, the CTA stops); 0 restores the default (2^22).  A tiny value
 * makes the waits expire on purpose, to test the error path from the host.
 */
int tfft_plan_set_wait_limit(tfft_plan plan, uint32_t polls);

/*
 * Timing hook: record caller-created CUDA events (cudaEvent_t as void*) on
 * the execution stream around every launch of the following tfft_execute()
 * calls: events[k] before launch k and events[n] after the last, n =
 * tfft_plan_num_launches().  count must be >= n + 1.  count = 0 removes the
 * hook.  The events stay owned by the caller.
 */
int tfft_plan_set_launch_events(tfft_plan plan, void *const *events, int count);

/*
 * Batched persistent executor: the fused transforms (one direction) of many
 * independent complex-to-complex plans -- each with its own shape and
 * virtual grid -- run by ONE kernel launch.  The launch's CTAs take the tiles
 * of every pass of every transform from a shared queue, segment by segment
 * (segment = one pass of one transform) in pass-major order.  A tile of
 * pass k of a transform waits (bounded,
 * ~2 s, then the device status word gets TFFT_DEVICE_ETIMEOUT = 1 and the
 * launch stops) until every tile of pass k-1 of the same transform is done.
 *
 *   tfft_batch_create   plans (host objects, bound before tfft_batch_bind)
 *   tfft_batch_state_bytes / tfft_batch_bind
 *                       caller-allocated device state; the in / out / work
 *                       pointers of every transform are fixed at bind time
 *                       (work[t] may be NULL: input t is then scratch)
 *   tfft_batch_execute  one memset of the queue counters + one kernel launch,
 *                       stream-ordered, no allocation and no host sync (so a
 *                       CUDA graph can capture it) -- or, with the stream
 *                       executor (tfft_batch_set_executor), every transform's
 *                       own pass kernels on forked streams, joined back
 *   tfft_batch_autotune picks, per pass kind and length, the fastest of the
 *                       compiled tile variants (elements per thread, tile
 *                       width / lines per group) by timing the whole batch
 *                       (`reps` runs per candidate); it runs the batch on the
 *                       bound buffers (their contents are overwritten) and
 *                       synchronises.  With TFFT_AUTOTUNE_CACHE set, choices
 *                       are read from / written to that file.  Then it
 *                       times the persistent kernel against the stream
 *                       executor with 1, 2, 3, 4, 6 and 8 streams and keeps
 *                       the fastest executor (cached as the line "-1 -1 K",
 *                       K = streams, 0 = persistent).
 * The paper has no batched executor; each transform follows its plan's steps.
 */
typedef struct tfft_batch_s *tfft_batch;
/* tfft_batch_bind's d_state must be 256-byte aligned (it holds TMA tensor maps). */
int tfft_batch_create(tfft_batch *batch, int count, const tfft_plan *plans, int sign);
int tfft_batch_destroy(tfft_batch batch);
int tfft_batch_state_bytes(tfft_batch batch, size_t *bytes);
int tfft_batch_bind(tfft_batch batch, void *d_state, size_t bytes, const void *const *ins,
                    void *const *outs, void *const *works, void *stream);
int tfft_batch_execute(tfft_batch batch, void *stream);
int tfft_batch_autotune(tfft_batch batch, int reps, void *stream);
/* Work items (tiles) and segments (transform passes) of one execute. */
int tfft_batch_num_items(tfft_batch batch, int64_t *items, int *segments);
/* Issue order: segment `index` (0 <= index < segments) is pass `pass` of
   transform `transform` (index into the create call's plans).  Host only. */
int tfft_batch_segment(tfft_batch batch, int index, int *transform, int *pass);
/* Executor tile variant chosen for passes of `kind` (0 contiguous, 1 strided) and length L. */
int tfft_batch_variant(tfft_batch batch, int kind, int L, int *variant);
/* Choose that variant by hand (one of the compiled candidates for kind and L,
   else TFFT_EINVAL) and rewrite the bound state; synchronises.  A strided
   TMA-staged variant applies to the segments whose layouts allow it (equal
   blocks, 16-byte aligned tile columns); the others of that length run the
   first plain variant. */
int tfft_batch_set_variant(tfft_batch batch, int kind, int L, int variant, void *stream);
/* Clock cycles a batch tile may wait for the previous pass (0: default ~2 s);
   a tiny value makes the waits expire on purpose (error-path tests). */
int tfft_batch_set_wait_limit(tfft_batch batch, long long cycles);
/* Status of the batch: the OR of its state's status word and its plans'
   (the stream executor's kernels report in their plans' states); `reset`
   clears all of them.  As tfft_plan_device_status otherwise. */
int tfft_batch_device_status(tfft_batch batch, int *status, int reset, void *stream);

/* Executors of tfft_batch_execute. */
enum {
  TFFT_BATCH_PERSISTENT = 0, /* one persistent kernel over every pass (the default) */
  TFFT_BATCH_STREAMS = 1     /* each transform's own pass kernels, on forked streams */
};
/* Choose the executor (host only; no GPU work).  TFFT_BATCH_STREAMS: the
   transforms are dealt, longest first, to the least-loaded of `nstreams`
   (1..16, at most the transform count) streams; on execute, an event on the
   caller's stream forks them, each runs its transforms' fused passes one after
   the other with the standalone kernels of their plans (so independent
   transforms overlap, and a transform's passes follow one another while its
   data may still be in L2), and the caller's stream waits for all of them.
   Capturable into one CUDA graph like the persistent launch.  The streams
   and events are created on the first execute (on the current device, which
   must be the plans' device; else TFFT_EINVAL) and destroyed with the batch.
   For TFFT_BATCH_PERSISTENT `nstreams` is ignored. */
int tfft_batch_set_executor(tfft_batch batch, int executor, int nstreams);
/* The executor in use and its stream count (0 for the persistent kernel). */
int tfft_batch_executor(tfft_batch batch, int *executor, int *nstreams);

/*
 * Fused transform whose scratch lives in a fixed device array inside this
 * library, for callers that may not allocate device memory -- e.g. a plugin
 * running in a host framework that owns all device memory through its own
 * allocator, where an extra cudaMalloc is forbidden or finds no memory.  The
 * paper has no counterpart; it is an interface convenience.
 *
 * Same result, bit for bit, as tfft_execute(plan, sign, TFFT_MODE_FUSED, in,
 * out, work, ...) with a caller-allocated workspace: the input is kept --
 * except by the complex-to-real backward of a TFFT_R2C plan (sign +1), which
 * uses its input as scratch here too and leaves it undefined.  Nothing is
 * allocated: the scratch is a static __device__ array of
 * TFFT_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library
 * holds until the process exits; a plan whose fused workspace
 * (tfft_plan_workspace_bytes) is larger is
 * rejected with TFFT_EWORKSPACE (message in tfft_last_error()).  The current
 * device must be the one the plan was bound on (else TFFT_EINVAL).
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress, with
 * the plan's device current); the first call on a device also loads the
 * library's module there, so make that first call before any stream capture.
 * All calls and all plans share the one array and it keeps the last call's
 * contents (every call overwrites what it reads, so nothing has to start at
 * zero); calls whose work overlaps on the GPU -- on different streams, or
 * from different threads -- race on it.
 */
#define TFFT_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int tfft_execute_noalloc(tfft_plan plan, int sign, const void *in, void *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TFFT_H */

/*
 * gpspca.h - C ABI of the GB300 (sm_103a) generalized power method for sparse PCA.
 *
 * The operation (paper "Large-Scale Paralleled Sparse Principal Component
 * Analysis", Section 2 and Table 1): A is a p x n data matrix (p samples of n
 * variables, columns a_i).  For the four formulations
 *
 *   SL1  max_{x in S^p}   sum_i [ |a_i^T x| - gamma ]_+^2
 *   SL0  max_{x in S^p}   sum_i [ (a_i^T x)^2 - gamma ]_+
 *   BL1  max_{X in S^p_m} sum_j sum_i [ mu_j |a_i^T x_j| - gamma_j ]_+^2
 *   BL0  max_{X in S^p_m} sum_j sum_i [ (mu_j a_i^T x_j)^2 - gamma_j ]_+
 *
 * the library runs the generalized power iteration: T = A^T X (column sweep),
 * a per-entry soft (L1) or hard (L0) threshold at gamma that yields the
 * gradient direction G, the rank update Y = A G, and the projection back onto
 * the feasible set (x = y/||y|| on the sphere, X = Y (Y^T Y)^{-1/2} on the
 * Stiefel manifold).  The sparse loadings Z of Table 1's "Original form"
 * column are recovered from the last sweep.  Every step runs in this
 * library's CUDA kernels; there is no host fallback.
 *
 * Conventions shared by all entry points
 *  - Matrices are column-major.  Element (r, i) of A is data[i*ld + r].  A C
 *    array or torch tensor of shape [n][ld] (rows = variables) is this layout.
 *  - m is always the number of gamma values.  Block forms: m components,
 *    gamma[j] and mu[j] belong to component j.  Single-unit forms: m
 *    independent solves on the same A, one per gamma (a sparsity path), all
 *    starting from the same x0; X then has m unit columns, not orthonormal.
 *  - Return value: GPSPCA_OK (0) or a negative GPSPCA_E* code; the message of
 *    the calling thread's last error is returned by gpspca_last_error().
 *    Nothing aborts the process or traps the device.
 *  - Memory: A, x0 and every output buffer belong to the caller.  The library
 *    borrows them until gpspca_solve returns, or until gpspca_poll returns
 *    GPSPCA_OK for the ticket; the caller must not free or modify them before.
 *    The library allocates only its own workspace, counted against the
 *    context's budget (GPSPCA_ENOMEM when a solve would exceed it).
 */
#ifndef GPSPCA_H
#define GPSPCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Formulations of Table 1. */
typedef enum { GPSPCA_SL1 = 0, GPSPCA_SL0 = 1, GPSPCA_BL1 = 2, GPSPCA_BL0 = 3 } gpspca_form;

/* Storage type of A.  F64 solves compute in double; the others compute in
 * float with double objective, normalisation, Gram matrix and stopping test.
 * FP8_E4M3 stores q_ri with a per-column float scale s_i: a_ri = q_ri * s_i. */
typedef enum { GPSPCA_F32 = 0, GPSPCA_BF16 = 1, GPSPCA_FP8_E4M3 = 2, GPSPCA_F64 = 3 } gpspca_dtype;

/* Where a caller buffer lives.  HOST buffers are copied by the library
 * (host to device before the solve, device to host after it); pinned host
 * memory makes those copies asynchronous. */
typedef enum { GPSPCA_DEVICE = 0, GPSPCA_HOST = 1 } gpspca_location;

/* Return codes. */
#define GPSPCA_OK 0
#define GPSPCA_PENDING 1          /* gpspca_poll: ticket not finished yet */
#define GPSPCA_EINVAL (-1)        /* bad shape, pointer, gamma < 0, mu <= 0, m > p (block), m > 64 */
#define GPSPCA_ENOMEM (-2)        /* workspace would exceed the context budget, or allocation failed */
#define GPSPCA_ENONFINITE (-3)    /* A has a NaN/Inf entry (or one whose square overflows float) */
#define GPSPCA_ETIMEDOUT (-4)     /* a device-side wait gave up; the context stays usable */
#define GPSPCA_EDEGENERATE (-5)   /* block polar step met a rank-deficient Y; outputs hold the last valid X */
#define GPSPCA_ECUDA (-6)         /* a CUDA runtime call failed */
#define GPSPCA_ENOTFOUND (-7)     /* gpspca_poll: unknown or already collected ticket; gpspca_tune_load: no file */

/* Per-solve termination status, written to out->status[j]. */
#define GPSPCA_CONVERGED 0   /* |f_k - f_{k-1}| < tol * f_{k-1} */
#define GPSPCA_MAXIT 1       /* maxit sweeps done */
#define GPSPCA_ZERO 2        /* f_k == 0: every entry thresholded (or A == 0) */
#define GPSPCA_DEGENERATE 3  /* lambda_min(Y^T Y) <= 1e-12 lambda_max(Y^T Y) in the polar step */

/* Flags for gpspca_solve / gpspca_submit. */
#define GPSPCA_GAMMA_RELATIVE 1u  /* gamma[j] is relative: the device scales it to
                                     gamma[j]*max_i||a_i|| (L1) or (gamma[j]*max_i||a_i||)^2 (L0) */
#define GPSPCA_EAGER 2u           /* launch the same kernels one by one with a host-driven loop
                                     (one device->host read of the active count per sweep)
                                     instead of the cached CUDA graph with its device-side WHILE
                                     node: for profilers and debuggers that cannot follow
                                     conditional graph nodes.  Results are identical. */
#define GPSPCA_NO_TENSOR_CORES 4u /* run the CUDA-core fused sweep even where the tensor-core
                                     (tcgen05) sweep applies (bf16 storage, or float storage with
                                     a 16-byte aligned base and column stride, with m >= 6; such
                                     float storage with p >= 16384 rows for any m; other float
                                     layouts and fp8 storage with m >= 9) */
#define GPSPCA_TIME_T_PASS 16u    /* gpspca_time_sweep only: time the tensor-core sweep's first
                                     pass (T = A^T X with its X3 preparation and row-range
                                     combine) without the rank update; GPSPCA_EINVAL where the
                                     problem does not run the tensor-core sweep */
#define GPSPCA_INJECT_TIMEOUT 8u  /* test hook for callers' error handling: after the solve has
                                     run, its device state is marked as if a device-side wait had
                                     given up, so the call returns GPSPCA_ETIMEDOUT (no wait is
                                     made to expire); the context stays usable */

/* Largest m (components, or gamma values of a path) one solve accepts. */
#define GPSPCA_MAX_M 64

/* The data matrix A (p x n, column-major, leading dimension ld >= p).
 * The buffer must hold ld*n elements.  The fast load path wants the base
 * address 16-byte aligned and ld*sizeof(element) a multiple of 16; other
 * layouts run on a slower element-wise load path.  col_scale: FP8_E4M3 only,
 * n floats in the same location as data (NULL otherwise). */
typedef struct {
  const void* data;
  gpspca_dtype dtype;
  gpspca_location location;
  int64_t p, n, ld;
  const float* col_scale;
} gpspca_matrix;

/* Caller-allocated results, all in `location`.  Element type of X and Z is
 * double for F64 solves and float otherwise.
 *   X          p x m column-major (ld p): the iterate that produced the objective
 *   Z          n x m column-major (ld n): unit-norm (or all-zero) sparse loadings
 *   support    ceil(n/32) x m uint32 words (may be NULL): bit (i % 32) of word
 *              j*ceil(n/32) + i/32 is set iff Z[i, j] != 0
 *   objective  m doubles: per gamma (single-unit) or per component f_j (block;
 *              the block objective is their sum)
 *   iters      m int32: sweeps t = A^T x performed
 *   status     m int32: GPSPCA_CONVERGED / MAXIT / ZERO / DEGENERATE
 *   gamma_abs  m doubles (may be NULL): the absolute gamma used */
typedef struct {
  gpspca_location location;
  void* X;
  void* Z;
  uint32_t* support;
  double* objective;
  int32_t* iters;
  int32_t* status;
  double* gamma_abs;
} gpspca_out;

typedef struct gpspca_ctx gpspca_ctx;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * library's own workspace, and for gpspca_submit also the admitted
 * requests' matrices and outputs (0 = 90% of the device's free memory).
 * cuda_stream: a cudaStream_t to run on, or NULL for a stream the context
 * creates.  Section 3's host/device flow: the context owns device workspace
 * and launches every step on that stream. */
int gpspca_create(gpspca_ctx** ctx, int device, size_t hbm_budget_bytes, void* cuda_stream);

/* One synchronous solve (Section 2, Table 1).
 *   A       data matrix descriptor (device or host)
 *   form    GPSPCA_SL1 / SL0 / BL1 / BL0
 *   gamma   host array of m values >= 0 (absolute unless GPSPCA_GAMMA_RELATIVE)
 *   m       1 <= m <= GPSPCA_MAX_M; block forms also need m <= p
 *   mu      host array of m weights > 0 (block forms), or NULL for all 1;
 *           must be NULL or all 1 for single-unit forms
 *   tol     stop when |f_k - f_{k-1}| < tol * f_{k-1} (k >= 1)
 *   maxit   >= 1: at most maxit sweeps
 *   x0      optional p x m starting iterate (same location as A; float, or
 *           double for F64); projected on the feasible set (columns
 *           normalised, or the polar factor for block forms).  NULL: the
 *           largest-norm column (single-unit, ties to the lower index) or,
 *           for block forms, the PCA start: a seeded Rademacher sketch of m
 *           columns (SplitMix64, seed 0x5EED5EED5EED5EED), two projected
 *           power steps with A A^T and a Rayleigh-Ritz rotation
 *   flags   GPSPCA_GAMMA_RELATIVE | GPSPCA_EAGER | GPSPCA_NO_TENSOR_CORES, or 0
 *   out     result buffers
 * Returns GPSPCA_OK, GPSPCA_EDEGENERATE (outputs valid, see status), or an
 * error code (outputs undefined). */
int gpspca_solve(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                 const double* mu, double tol, int32_t maxit, const void* x0, uint32_t flags, gpspca_out* out);

/* One solve of a batch (gpspca_solve_batch): the arguments of gpspca_solve. */
typedef struct {
  gpspca_matrix A;
  gpspca_form form;
  const double* gamma;  /* m values */
  int32_t m;
  const double* mu;     /* NULL or m values */
  double tol;
  int32_t maxit;
  const void* x0;       /* NULL or a starting iterate, as for gpspca_solve */
  uint32_t flags;
  gpspca_out out;
} gpspca_request;

/* count independent solves (same arguments, ownership and results as
 * gpspca_solve, one request each) run concurrently: each on its own stream
 * and workspace (up to 8 at a time, in request order beyond that), so that
 * the latency-bound steps of one solve (reductions, the projection's small
 * eigenproblem) overlap the sweeps of the others.  Stream-ordered with the
 * context's stream: the batch starts after the work already enqueued on it,
 * and work enqueued on it afterwards starts after the whole batch.  Returns
 * when every solve has finished; rcs[i] (count entries, caller-owned)
 * receives solve i's result code.  The return value is GPSPCA_OK when every
 * solve returned GPSPCA_OK or GPSPCA_EDEGENERATE, else the first other code.
 * A host matrix shared by several requests of the batch (same data pointer,
 * dtype, shape, ld and col_scale) is copied to the device once, on the
 * context's stream before the batch starts, into a buffer the context keeps
 * (counted against the budget) for later batches.  Two or more single-unit
 * requests that are not grouped (below) and share one device matrix (same
 * data pointer, dtype, shape, ld and col_scale, the staged copy included)
 * take its column norms from one pass the batch makes for them on the
 * context's stream, each copying them with its own non-finite check; their
 * results are bit-identical to solo solves.  Four or more single-unit
 * requests with one component and the same storage type, form, shape,
 * column stride and alignment (device matrices; not GPSPCA_EAGER) run as a
 * group of up to 256: each step of their solves is one kernel launch for
 * all of them.  A member's sweep sums over fewer column slabs than a solo
 * solve's, so it agrees with a solo solve to float rounding; its bits do
 * not depend on the group's size or other members. */
int gpspca_solve_batch(gpspca_ctx* ctx, int32_t count, const gpspca_request* reqs, int32_t* rcs);

/* Asynchronous copy of a host matrix to device memory the caller owns, so
 * that the copy of the next problem overlaps the solves of this one (no
 * counterpart in the paper: its host/device flow of Section 3 copies A before
 * the iterations).
 *   host  GPSPCA_HOST matrix (page-locked memory for the copy to overlap
 *         anything; pageable memory is copied too, without overlap)
 *   dst   GPSPCA_DEVICE matrix of the same dtype, p and n; its own ld >= p
 *         (the copy re-strides when the two ld differ); FP8 storage: both
 *         col_scale arrays (host / device, n floats) are copied as well
 * The copy runs on a stream of the context's own, after the work already
 * enqueued on the context's stream, and the call returns at once.  Every
 * later gpspca_solve, gpspca_solve_batch, gpspca_submit, gpspca_solve_deflated,
 * gpspca_project, gpspca_time_sweep and gpspca_tune of this context whose
 * matrix has dst's data pointer waits on the device for the copy of the
 * latest upload to that pointer (gpspca_sweep_static, which has no context,
 * does not).  The host memory must stay unchanged until the copy has
 * finished: a synchronous call that reads dst has returned, or a submitted
 * one has been polled to completion.  dst must not be written to again, by
 * an upload or otherwise, while a solve that reads it is still running.  The context remembers the last 16
 * destinations.  Returns GPSPCA_OK, GPSPCA_EINVAL (locations, shapes or types
 * that do not match, NULL pointers) or GPSPCA_ECUDA. */
int gpspca_upload(gpspca_ctx* ctx, const gpspca_matrix* host, const gpspca_matrix* dst);

/* Several sparse components with a single-unit formulation (form SL1 or
 * SL0), by projection deflation: component j (0 <= j < m) is the single-unit
 * solve with gamma[j] (as gpspca_solve with one gamma value, same start and
 * stopping rule) on the deflated matrix
 *   A_0 = A,   A_j = A_{j-1} - u_j z_j^T,   u_j = A_{j-1} z_j,
 * i.e. A_j = A_{j-1} (I - z_j z_j^T) with z_j the unit loading (Z column) of
 * component j, so that A_j z_j = 0.  The paper extracts several single-unit
 * components (Section 4.1, Fig. 3, m = 5) without naming the deflation; this
 * is the reading taken.  With GPSPCA_GAMMA_RELATIVE, gamma[j] is relative to
 * the largest column norm of A_{j-1}.
 *
 * A is not modified.  The library deflates a working copy (float; double for
 * F64 storage, whose solves compute in double; bf16 / fp8 storage is widened
 * to float, fp8 times its column scale), held only during the call and
 * counted against the budget (p x n elements of the working type), touching
 * only the support columns of each z_j.  Results as for gpspca_solve with m
 * entries: column j of X, Z and support, objective[j] (f of component j on
 * A_{j-1}), iters[j], status[j] and gamma_abs[j] belong to component j.  A
 * component with status ZERO deflates nothing.  Flags: GPSPCA_GAMMA_RELATIVE,
 * GPSPCA_EAGER, GPSPCA_NO_TENSOR_CORES.  Returns when every component is done
 * (GPSPCA_EINVAL for a block form). */
int gpspca_solve_deflated(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                          double tol, int32_t maxit, uint32_t flags, gpspca_out* out);

/* Scores of samples on sparse loadings: S = B Z.  The paper maps every
 * sample (training and test) into the subspace of the learned components
 * before classifying (Section 4.2); with the loadings Z of a solve (n x m,
 * column-major, ld n) and samples B (q x n: q samples of the same n
 * variables, column-major like A, any storage type; fp8 with its column
 * scales), S (q x m, column-major, ld q) gets column j = sum_i Z[i, j] b_i.
 * Only the columns of B in the support of each loading are read, so the cost
 * is q * |supp z_j| elements per component.  Z and S are double for F64
 * storage and float otherwise; sums in double-float (double for F64).
 * B, Z and S are all in B's location (device, or host: copied by the
 * library).  Returns when S is written.  GPSPCA_EINVAL for m outside
 * [1, GPSPCA_MAX_M], NULL pointers or a bad shape. */
int gpspca_project(gpspca_ctx* ctx, const gpspca_matrix* B, const void* Z, int32_t m, void* S);

/* Asynchronous form of gpspca_solve for many concurrent requests.  The
 * request is queued; a scheduler thread admits it into one of 8 slots (each
 * with its own stream and workspace) when its HBM footprint fits the context
 * budget next to the solves already running, and launches it there as a
 * whole solve (the cached CUDA graph of its geometry), so requests that
 * arrive while others run overlap with them on the device.  The footprint is
 * the request's own device bytes (its matrix, fp8 scales and outputs) plus
 * the workspace of its solve; both stay reserved until the request
 * completes.  A request that does not fit waits for running ones to finish;
 * one whose matrix and outputs alone exceed the budget returns GPSPCA_ENOMEM
 * here (one that cannot fit even alone, workspace included, completes with
 * GPSPCA_ENOMEM).  Same arguments and ownership as gpspca_solve (A and out
 * must be in device memory); *ticket receives the request id. */
int gpspca_submit(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                  const double* mu, double tol, int32_t maxit, uint32_t flags, gpspca_out* out,
                  uint64_t* ticket);

/* Wait up to wait_us microseconds (0 = just look, < 0 = until done) for a
 * ticket.  Returns GPSPCA_PENDING, or the ticket's result code (as
 * gpspca_solve would return it) once, after which the ticket is forgotten. */
int gpspca_poll(gpspca_ctx* ctx, uint64_t ticket, int32_t wait_us);

/* Autotuner (the paper has no counterpart; it picks how the sweep of
 * Section 2 / Table 1 is laid out on the GPU, not what it computes).  Times
 * every candidate sweep layout for this problem (the tensor-core sweep where
 * its storage type allows it, and every grouping of the components into
 * CUDA-core passes of at most 8, 5, 4, 2 or 1 in clusters of 1, 2, 4 or 8
 * CTAs that fits on chip): for each, the start and
 * projection as gpspca_solve runs them, one warm-up sweep, then `reps`
 * sweeps between CUDA events.  The fastest layout is remembered for this
 * shape (storage type, single-unit or block form, m, p, n, ld, alignment,
 * tensor-core permission, SM count) by the context, and later solves of the
 * shape use it; results are discarded.  *n_candidates receives the number of
 * layouts timed, *ms_best the fastest one's milliseconds per sweep and
 * *ms_default the planner's own choice's.  Arguments as gpspca_time_sweep.
 * The tuned layout changes only the order of the float partial sums, not the
 * iteration. */
int gpspca_tune(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                const double* mu, uint32_t flags, int32_t reps, int32_t* n_candidates, double* ms_best,
                double* ms_default);

/* Write the context's tuned layouts to a text file (a "gpspca-tune 1" line,
 * then one "shape TAB layout TAB milliseconds" line per shape).  GPSPCA_EINVAL
 * if the file cannot be written. */
int gpspca_tune_save(gpspca_ctx* ctx, const char* path);

/* Merge the tuned layouts of a file written by gpspca_tune_save into the
 * context.  A layout is used only where the planner still offers it on this
 * device (otherwise the default plan runs).  GPSPCA_ENOTFOUND if the file
 * cannot be read, GPSPCA_EINVAL if it is not such a table (nothing merged). */
int gpspca_tune_load(gpspca_ctx* ctx, const char* path);

/* Measurement aid (the paper has no counterpart): prepare a solve (start
 * and projection, as gpspca_solve
 * does), then time `reps` back-to-back launches of the fused sweep of one
 * iteration (every component pass) on the context's stream with CUDA events.
 * *ms_per_sweep receives the mean milliseconds per sweep.  A must be on the
 * device or the host as for gpspca_solve; results are discarded. */
int gpspca_time_sweep(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                      const double* mu, uint32_t flags, int32_t reps, double* ms_per_sweep);

/* Seeded synthetic input (not part of the method): a planted-spike matrix
 * drawn on the device, for workloads whose requests bring their own data
 * (the serving benchmark).  Writes A (p x n, column-major, leading dimension
 * ld >= p; float32 or bfloat16, device memory At) with
 *   A[r, i] = z_ri + [column i in the support of spike j] s_i theta_j/sqrt(s) u_j[r],
 * z and u_j standard normal, j < k <= 64 spikes on disjoint supports of
 * expected size s = max(1, round(support_frac * n)) (k * support_frac <= 1),
 * Rademacher signs s_i.  Every value comes from Philox4x32-10 (Salmon et al.,
 * SC'11) under key = seed, with Box-Muller in float32: noise rows 4b..4b+3 of
 * column i from counter (b, i_lo, i_hi, 0), u_j rows from (b, j, 0, 1), the
 * spike and sign of column i from words 0 and 1 of (i_lo, i_hi, 0, 2).
 * theta: host array of k values.  Asynchronous on cuda_stream.  Returns
 * GPSPCA_OK or GPSPCA_EINVAL / GPSPCA_ECUDA. */
int gpspca_synth_spikes(void* At, gpspca_dtype dtype, int64_t p, int64_t n, int64_t ld, int32_t k,
                        const double* theta, double support_frac, uint64_t seed, void* cuda_stream);

/* Measurement aid (the paper has no counterpart): the number of kernel
 * launches of one solve of this problem with the layout gpspca_solve would
 * pick, as counts[0] before the iterations (start, norms, projection, and
 * for block forms the power steps of the start), counts[1] per iteration
 * (the sweep's kernels, its reduction and its finish step) and counts[2]
 * after them (the loadings).  A solve that runs k iterations launches
 * counts[0] + k counts[1] + counts[2] kernels.  Arguments as
 * gpspca_time_sweep; nothing is launched. */
int gpspca_plan_launches(gpspca_ctx* ctx, const gpspca_matrix* A, gpspca_form form, const double* gamma, int32_t m,
                         const double* mu, uint32_t flags, int32_t counts[3]);

/* One fused single-unit sweep that allocates no memory.  The paper has no
 * counterpart: this entry point is for callers that cannot allocate device
 * memory at the moment they need a sweep, e.g. because another framework's
 * caching allocator holds the free HBM, because the call sits in a
 * latency-bound loop where an allocation could synchronise the device, or
 * because it runs where allocation is forbidden.  No context is needed.
 *
 * For a float32 matrix A in device memory and a device iterate x (p floats,
 * used as given), it computes on the device: t = A^T x (n floats), the
 * single-unit objective f at x (one double: sum of [|t_i| - gamma]_+^2 for
 * SL1, of [t_i^2 - gamma]_+ for SL0) and x_next = A g / ||A g|| (p floats; all
 * zero when every entry is thresholded), where g is the SL1 or SL0 gradient
 * factor at gamma (absolute).  All outputs are caller-owned device memory.
 * cuda_stream (NULL: the legacy default stream) must belong to the current
 * device; the call synchronises with it and returns when the results are
 * ready, so it cannot itself run under stream capture.
 *
 * Scratch lives in file-scope device arrays of fixed size (6 MiB: the
 * per-cluster partials of y, up to 160 clusters x p floats) that every GPU
 * loading the library keeps until the process exits.  Limit: p <= 8192;
 * a larger p returns GPSPCA_EINVAL naming the limit.  The arrays are shared
 * by every call and keep the last call's contents (everything a call reads
 * is rewritten by it first): calls are serialised inside the library, and
 * calls that overlapped on the GPU (e.g. from other processes) would race.
 * The first call on a device resolves the arrays' device addresses
 * (cudaGetSymbolAddress) for that device; make it before any stream capture
 * on the device.  A NaN or infinity in A or x (or an overflow of t, f or
 * ||A g||) returns GPSPCA_ENONFINITE.  No cudaMalloc, cudaFree or allocating
 * library routine is called. */
int gpspca_sweep_static(const gpspca_matrix* A, gpspca_form form, double gamma, const float* x, float* x_next,
                        float* t, double* objective, void* cuda_stream);

/* Finish queued work, free every workspace buffer and the context. */
int gpspca_destroy(gpspca_ctx* ctx);

/* Message for the calling thread's last error ("" if none). */
const char* gpspca_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GPSPCA_H */

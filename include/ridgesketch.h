/*
 * ridgesketch.h -- C ABI of the GB300 sketch-and-project ridge regression solver.
 *
 * The library solves ridge regression (Section 2.1, eq. (1)):
 *     min_w 1/2 ||X w - y||^2 + lambda/2 ||w||^2
 * through the linear system A w = b of eq. (4), in primal form
 *     A = X^T X + lambda I,  b = X^T y            (eq. (2), m = d)
 * or dual form
 *     A = X X^T + lambda I,  b = y,  w = X^T alpha  (eq. (3), m = n),
 * with the sketch-and-project method with momentum (Algorithm 2, Section 6.3):
 *     r_S   = S_k^T r^k
 *     delta = least-norm solution of (S_k^T A S_k) delta = r_S          (eq. (14))
 *     w^{k+1} = (1 + beta_k) w^k - beta_k w^{k-1} - gamma_k S_k delta
 *     r^{k+1} = (1 + beta_k) r^k - beta_k r^{k-1} - gamma_k A S_k delta  (eq. (53))
 * starting from w^{-1} = w^0 = 0, r^{-1} = r^0 = -b, and stopping once
 * ||r^k|| / ||r^0|| <= tol (the stopping rule of Section 3).
 *
 * Sketches (Section 4): Gaussian, Subsample, Count, SubCount, SRHT. Momentum
 * (Section 8.1): none, constant, theoretical ("increasing", eq. (66)), heuristic
 * (eq. (67)). Every step of an iteration runs in this library's CUDA kernels on
 * one GPU.
 *
 * Conventions for every entry point:
 *  - Return RS_OK (0) on success, another rs_status on failure; no C++ exception
 *    crosses the ABI. A failure message is available from rs_last_error(ctx)
 *    (or rs_last_error(NULL) for failures without a context, e.g. in rs_create).
 *  - Pointers flagged "on_device" are CUDA device pointers of the context's device;
 *    all others are host pointers. Input buffers are only read during the call
 *    (the library copies what it keeps); output buffers are caller-owned and
 *    written during the call.
 *  - Row-major dense layouts; sizes are element counts.
 *  - All work of a context is issued on the context's stream (rs_opts.cuda_stream,
 *    or a blocking stream the library creates, whose work orders after the work
 *    issued before it on the legacy default stream). Device inputs written on any
 *    other stream must be complete, or that stream ordered before the context's
 *    stream, when the call starts. Calls on one context must not overlap.
 */
#ifndef RIDGESKETCH_H
#define RIDGESKETCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rs_ctx rs_ctx; /* opaque; owned by the library until rs_destroy */

typedef enum {
  RS_OK = 0,
  RS_EINVAL = 1,     /* invalid argument (null pointer, bad size, bad enum) */
  RS_ENOMEM = 2,     /* device or host allocation failed */
  RS_ECUDA = 3,      /* a CUDA runtime call failed */
  RS_ENUMERIC = 4,   /* NaN or Inf in the residual */
  RS_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  RS_ENOTCONV = 6,   /* max_iters reached before tol; outputs are still valid */
  RS_EUNSUPPORTED = 7 /* combination of options this build does not implement */
} rs_status;

typedef enum { RS_PRIMAL = 0, RS_DUAL = 1 } rs_form;

/* Section 4.1 (Gaussian, Subsample), 4.2 (Count, SubCount), 4.3 (SRHT). */
typedef enum {
  RS_GAUSSIAN = 0,
  RS_SUBSAMPLE = 1,
  RS_COUNT = 2,
  RS_SUBCOUNT = 3,
  RS_SRHT = 4
} rs_sketch;

/* Section 8.1: none (gamma = 1, beta = 0), constant (gamma_c, beta_c),
 * theoretical increasing momentum (eq. (66) with eqs. (38), (40)), heuristic
 * (eq. (67): gamma = 1 with the theoretical beta_k). */
typedef enum {
  RS_MOM_NONE = 0,
  RS_MOM_CONST = 1,
  RS_MOM_THEORY = 2,
  RS_MOM_HEURISTIC = 3
} rs_mom_kind;

typedef enum {
  RS_F64 = 0,
  RS_F32 = 1,
  RS_BF16 = 2 /* CSR values only (bfloat16, 2 bytes); products widen them exactly */
} rs_dtype;

typedef enum {
  RS_PLAIN_FP64 = 0, /* every product and update in FP64 */
  RS_MIXED = 1       /* A, A S in FP32 (A formed with FP32 accumulation), FP64
                        vectors, FP64 true residual through X every refresh_every
                        iterations and before declaring convergence */
} rs_precision;

typedef struct {
  int32_t kind;        /* rs_mom_kind */
  int32_t uncapped;    /* heuristic only: 1 = closed form of eq. (50) for all k */
  double eta;          /* eta of eq. (66); default 0.995 */
  double beta_switch;  /* beta at which eta switches to 1; default 0.5 */
  double gamma_c;      /* constant mode step size; default 1.0 */
  double beta_c;       /* constant mode momentum; default 0.5 */
} rs_mom;

/*
 * Design matrix X, n x d: dense row-major (is_csr = 0: val holds n*d values of
 * dtype RS_F64 or RS_F32) or CSR (is_csr = 1: rowptr[n + 1] with rowptr[0] = 0 and
 * rowptr[n] = nnz, colidx[nnz] in [0, d), val[nnz] of dtype RS_F64, RS_F32 or
 * RS_BF16; column indices need not be sorted within a row, duplicates add up).
 * A CSR X runs matrix-free (A = X^T X + lambda I is never formed; A V =
 * X^T (X V) + lambda V, Section 2), primal form, subsample / count / subcount
 * sketches; inconsistent CSR arrays give RS_EINVAL (checked on the device before
 * any use). The arrays are copied; n, d < 2^31.
 */
typedef struct {
  int32_t is_csr;       /* 0 dense, 1 CSR */
  int32_t dtype;        /* rs_dtype of val */
  int64_t n, d;         /* rows (samples), columns (features) */
  int64_t nnz;          /* CSR: stored entries */
  const void* val;      /* dense: n*d values, row-major; CSR: nnz values */
  const int64_t* rowptr;/* CSR: n + 1 row offsets */
  const int32_t* colidx;/* CSR: nnz column indices */
  int32_t on_device;    /* 1 if val (and rowptr/colidx) are device pointers */
} rs_matrix;

typedef struct {
  int32_t precision;     /* rs_precision; default RS_PLAIN_FP64 */
  int32_t refresh_every; /* RS_MIXED: FP64 true-residual period in iterations; default 50.
                            A chunk shorter than the period shortens it to the chunk */
  int64_t sub_s;         /* SubCount sample size s (multiple of tau, <= m); 0 = rule of
                            Section 4.2: k = 10 if 10 tau <= m else floor(m/tau), s = k tau */
  void* cuda_stream;     /* cudaStream_t to issue work on; NULL = library-owned stream */
  int32_t device;        /* CUDA device ordinal; default 0 */
  int32_t chol_fp64;     /* RS_MIXED only: 1 = the small solve in FP64 (default): S^T A S
                            (summed from the FP32 A) is factored by an FP64 Cholesky and
                            its pseudo-inverse formed and applied in FP64; 0 = FP32 (M^+ by
                            FP32 sweeps). RS_PLAIN_FP64 always works in FP64 */
  int64_t chunk;         /* iterations per device-side chunk: the sketched systems of a
                            chunk are formed and factored ahead in batched launches, and
                            the chunk's iterations follow (RS_MIXED: one launch of the
                            persistent kernel per refresh period, an FP64 refresh after
                            each). 0 = 600 (128 for plain FP64 CSR X). RS_MIXED rounds it up
                            to a whole number of refresh periods; every kind reduces it so
                            that the chunk's buffers stay within a quarter of the
                            free device memory, at least 4 GB and at most 16 GB */
  int32_t setup_tc;      /* RS_MIXED, primal, FP32 X: 1 = form X^T X on the tensor cores
                            (TF32 inputs, FP32 accumulation; default), 0 = FP32 CUDA cores */
  int32_t iter_ctas;     /* subsample / count / subcount: CTAs of the persistent iteration
                            kernel that spreads the rows of w and r over the GPU (rounded
                            down to a multiple of 8); 0 = every SM (default); -1 = use the
                            single-cluster iteration kernel instead */
  int64_t spin_limit_ns; /* bound, in ns of the GPU's global timer, of every wait of the
                            persistent iteration kernel on other CTAs (its all-reduce) and
                            on its copies; a wait that runs out ends the solve with
                            RS_ETIMEOUT and leaves the context usable. 0 = 2 s */
  int64_t stall_ns;      /* fault injection for tests of those waits: CTA 0 of the
                            persistent iteration kernel publishes its first partials this
                            many ns late in every launch; 0 = none (default) */
  const char* tune_cache;/* batch autotuner: file that keeps its choices (read when it
                            exists, written after a measurement); NULL = none. Read by
                            rs_create_batch only; the string is copied */
} rs_opts;

/* Fill *o with the defaults listed above. */
void rs_default_opts(rs_opts* o);
/* Fill *m with the defaults of the given momentum kind (rs_mom_kind). */
void rs_default_mom(rs_mom* m, int32_t kind);

/*
 * Create a solver context: copies X and y to the device, forms A and b
 * (eqs. (2)-(4)) on the device, and prepares the buffers of the iteration.
 *   X       design matrix (see rs_matrix); X is kept on the device for the dual
 *           recovery w = X^T alpha and for RS_MIXED true residuals.
 *   y       n targets (FP64); device pointer if y_on_device.
 *   lambda  regularisation, > 0.
 *   form    rs_form.
 *   sketch  rs_sketch.
 *   tau     sketch size, 1 <= tau <= m (SRHT: tau <= 2^ceil(log2 m)); 0 selects
 *           ceil(m^(2/3)) (the rule of thumb of Section 8.1).
 *   mom     momentum parameters (NULL = no momentum).
 *   seed    seed of the counter-based sketch generator.
 *   opts    options (NULL = defaults).
 *   out     receives the context; NULL on failure.
 */
rs_status rs_create(const rs_matrix* X, const double* y, int32_t y_on_device, double lambda,
                    int32_t form, int32_t sketch, int64_t tau, const rs_mom* mom,
                    uint64_t seed, const rs_opts* opts, rs_ctx** out);

/*
 * Run the iteration from w^0 = 0 (every call restarts) until
 * ||r^k|| / ||r^0|| <= tol or k = max_iters.
 *   w_out      d weights (primal w, or X^T alpha for the dual), caller-owned;
 *              device pointer if w_on_device; may be NULL.
 *   hist_out   max_iters + 1 host doubles: hist[k] = ||r^k|| / ||r^0|| for
 *              k = 0..iters (RS_MIXED: entries at true-residual refreshes hold the
 *              FP64 true residual); may be NULL.
 *   iters_out  number of iterations run; may be NULL.
 * Returns RS_ENOTCONV if max_iters was reached first (outputs valid), RS_ENUMERIC
 * if the residual became NaN/Inf.
 */
rs_status rs_solve(rs_ctx* ctx, double tol, int64_t max_iters, double* w_out,
                   int32_t w_on_device, double* hist_out, int64_t* iters_out);

/*
 * Kernel ridge regression with the Gaussian kernel (Section 2.2): the n x n kernel
 * matrix K_ij = exp(-||p_i - p_j||^2 / (2 sigma^2)) (eq. (Gausskernel)) of the rows of
 * P, and the system K (K + lambda I) alpha = K y (eq. (kernelridge)), A = K^T (K +
 * lambda I), b = K^T y, solved like any other (rs_solve: w_out receives alpha, n
 * entries; predictions are K alpha).
 *   P       n x d points, dense row-major, RS_F64 or RS_F32 (host or device, copied)
 *   y       n targets (FP64); sigma > 0, lambda > 0; the rest as for rs_create
 * RS_PLAIN_FP64: K from the differences of the points in FP64, A by an FP64 product.
 * RS_MIXED: K on the tensor cores (TF32 products of the points, FP32 accumulation in
 * tensor memory, the exponential in the epilogue), FP32 K taken as the problem's data;
 * A = K^T K on the tensor cores; the FP64 refresh forms K^T (K w) + lambda K w - b with
 * FP64 sums over that K. Errors as rs_create.
 */
rs_status rs_create_kernel(const rs_matrix* P, const double* y, int32_t y_on_device, double lambda,
                           double sigma, int32_t sketch, int64_t tau, const rs_mom* mom,
                           uint64_t seed, const rs_opts* opts, rs_ctx** out);
/* The kernel matrix of a kernel ridge context (n x n doubles, host, row-major). */
rs_status rs_get_kernel(rs_ctx* ctx, double* K_out);

/*
 * Conjugate Gradients (Hestenes and Stiefel, 1952) on the same system A w = b: the
 * direct competitor of the paper's Experiment 3 (Section 8.3), for time-to-tolerance
 * comparisons on the same context. The sketch settings are not used. Dense A: the
 * formed A (FP64; RS_MIXED: the FP32 A with float-pair products and the FP64 true
 * residual through X every refresh_every iterations, which also decides convergence,
 * and CG restarts from it: iterative refinement with an inner CG on the FP32 A);
 * CSR X: A p = X^T (X p) + lambda p with FP64 sums over the stored values. Starts
 * from w = 0. Arguments, outputs and status codes as for rs_solve (hist_out: the
 * relative residual of every iteration, FP64-checked ones at the refreshes);
 * rs_timings reports its solve time.
 */
rs_status rs_solve_cg(rs_ctx* ctx, double tol, int64_t max_iters, double* w_out,
                      int32_t w_on_device, double* hist_out, int64_t* iters_out);

/* Free every resource of the context. NULL is accepted. The device memory of the
 * contexts comes from one stream-ordered pool per device that keeps freed blocks
 * for the next context (no cudaMalloc / cudaFree per context once warm). */
void rs_destroy(rs_ctx* ctx);

/* Return the pool's unused device memory on `device` to the driver (memory of live
 * contexts stays). RS_EINVAL for a device ordinal outside [0, 64). */
rs_status rs_trim_memory(int32_t device);

/* Message of the last failure on ctx (ctx = NULL: last failure without a context).
 * The string is owned by the library and valid until the next call on ctx. */
const char* rs_last_error(const rs_ctx* ctx);

/* Problem sizes of a context: m (system size), tau, s (SubCount sample size, else 0),
 * k_sum (SubCount sum size, else 0), m_pad (SRHT padded size 2^ceil(log2 m), else 0). */
rs_status rs_get_dims(const rs_ctx* ctx, int64_t* m, int64_t* tau, int64_t* s,
                      int64_t* k_sum, int64_t* m_pad);

/*
 * The chunking of a context (measurement and tests): *chunk = iterations per chunk
 * (slots whose sketched systems phase 1 forms in one batch), *refresh_every = the
 * FP64 refresh period (RS_MIXED; 0 for plain FP64), *fused_potri = 1 when M^+ is
 * formed by the one-kernel factor, inverse and product. Any pointer may be NULL.
 */
rs_status rs_chunking(const rs_ctx* ctx, int64_t* chunk, int32_t* refresh_every,
                      int32_t* fused_potri);
/* Launch shape of the fused iteration kernel of a context: ctas CTAs owning q rows
 * each of w and r (persistent kernel over the GPU), or ctas = q = 0 when the chunk's
 * iterations run on one thread-block cluster (Gaussian; or the slices do not fit
 * shared memory; or rs_opts.iter_ctas = -1). Outputs may be NULL. */
rs_status rs_iter_plan(const rs_ctx* ctx, int32_t* ctas, int64_t* q);

/*
 * Sketch of iteration k as drawn by the device generator (parity hook), host outputs:
 *   RS_SUBSAMPLE: idx[j] = C_j, j < tau
 *   RS_COUNT:     bucket[i], sign[i] for i < m
 *   RS_SUBCOUNT:  idx[p] = C_p, sign[p], bucket[p] = p / k_sum for p < s
 *   RS_SRHT:      idx[j] = C_j in [0, m_pad), j < tau; sign[i], i < m
 *   RS_GAUSSIAN:  RS_EINVAL (use rs_dump_gaussian)
 * Unused outputs may be NULL.
 */
rs_status rs_dump_sketch(rs_ctx* ctx, int64_t k, int32_t* idx, int8_t* sign, int32_t* bucket);

/* Gaussian sketch S of iteration k as an m x tau row-major host array (parity hook). */
rs_status rs_dump_gaussian(rs_ctx* ctx, int64_t k, double* S);

/*
 * Iteration state (w^k, w^{k-1}, r^k, r^{k-1}, k), host arrays of m doubles
 * (for the dual form these are alpha and its residual). rs_set_state replaces the
 * state so that rs_probe_step or rs_step continue from it (checkpoint/resume).
 */
rs_status rs_get_state(rs_ctx* ctx, double* w, double* w_prev, double* r, double* r_prev,
                       int64_t* k);
rs_status rs_set_state(rs_ctx* ctx, const double* w, const double* w_prev, const double* r,
                       const double* r_prev, int64_t k);

/*
 * Parity hook: for the current state and iteration k, compute the sketched system
 * M = S_k^T A S_k (tau x tau, row-major), r_S = S_k^T r^k and delta (eq. (14)) on
 * the device and copy them to the host without changing the state. Any output may
 * be NULL.
 */
rs_status rs_probe_step(rs_ctx* ctx, double* M, double* r_S, double* delta);

/* Run n_iters iterations from the current state (no stopping test, no refresh);
 * hist_out (n_iters entries, may be NULL) receives ||r^{k+1}|| / ||r^0||. */
rs_status rs_step(rs_ctx* ctx, int64_t n_iters, double* hist_out);

/* FP64 true relative residual ||A v - b|| / ||b|| of v (m host doubles: w for the
 * primal, alpha for the dual), evaluated through X without forming A. */
rs_status rs_true_residual(rs_ctx* ctx, const double* v, double* rel_out);

/* Device time of the last rs_solve (ms), split into setup (forming A, b in
 * rs_create; for FP32 X on the device it includes the context's copy of X, and for
 * FP32 X in host memory with n >= 16384 on the mixed primal path it includes the
 * upload of X, which that setup overlaps with its arithmetic) and iterations. Either
 * pointer may be NULL. */
rs_status rs_timings(const rs_ctx* ctx, double* setup_ms, double* solve_ms);

/* Per-kernel device time of the iteration (measurement hook). */
typedef struct {
  char name[32];      /* kernel group: "gen", "sa_rows", "msys", "chol", "update", "refresh", ... */
  int64_t launches;   /* launches timed */
  double ms;          /* mean device time per launch (CUDA events on the context stream) */
  double bytes;       /* algorithmic bytes moved per launch (inputs read once + outputs written) */
  double flops;       /* algorithmic floating-point operations per launch */
  int64_t iters;      /* iterations covered by the launches (fused chunk kernel), else launches */
} rs_kernel_stat;

/*
 * Continue the iteration from the current state for `reps` iterations, launching
 * each kernel group of an iteration separately between CUDA events on the context
 * stream, and report per group the mean time per launch and the algorithmic bytes
 * and flops of one launch. Writes at most `cap` entries to out and their number to
 * *n_out. The state advances by `reps` iterations (no stopping test).
 */
rs_status rs_profile_iteration(rs_ctx* ctx, int64_t reps, rs_kernel_stat* out, int32_t cap,
                               int32_t* n_out);

/*
 * out = X^T (X v) for a dense FP32 X, with FP64-accurate sums (the product the
 * library uses for true residuals of the primal form), WITHOUT ALLOCATING ANY MEMORY.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc or any allocating routine -- for example code running inside a
 * region where allocation is forbidden (a real-time loop with a no-allocation
 * policy, a host framework that owns all device memory and forbids others to
 * allocate, a program that must not change its memory footprint after start-up).
 *   X      n x d row-major FP32, device pointer (exact data; not modified)
 *   v      d FP64, device pointer
 *   out    d FP64, device pointer, caller-owned, overwritten
 *   stream cudaStream_t to run on (NULL = default stream)
 * Limits: 1 <= n, 1 <= d <= 4096 (RS_EINVAL beyond, with a message from
 * rs_last_error(NULL)). Work space: a fixed 2 MiB device array inside the library
 * (64 x 4096 doubles), held by every GPU that loads the library until the process
 * exits. The first call on a device looks up that array's device address (with the
 * device current), so make the first call before any stream capture. All calls share
 * the array: calls that overlap on the GPU (other streams, other host threads) race
 * and give wrong results; serialise them. Every entry the kernels read is written by
 * the same call, so no clearing is needed between calls. The array's address is
 * cached per device for the life of the process: after cudaDeviceReset on a device,
 * that address (like every other device state of the library on that device) is no
 * longer valid, so do not call this entry point on that device again. Runs
 * asynchronously on `stream`; returns RS_ECUDA if a launch fails.
 */
rs_status rs_gram_apply_noalloc(const float* X, int64_t n, int64_t d, const double* v,
                                double* out, void* stream);

/*
 * Batch of P independent primal ridge problems with nrhs right-hand sides each,
 * solved together: the iterations of every problem and right-hand side of a chunk
 * run in one persistent launch (one CTA per problem), the right-hand sides of a
 * problem sharing its sketches, S^T A and the small system's pseudo-inverse
 * (Algorithm 2, eq. (53), applied to A_p W = B_p column by column).
 *   P        number of problems, >= 1
 *   Xs       P dense matrices (rs_matrix, is_csr = 0; FP32 for RS_MIXED), copied
 *   Ys       P pointers; Ys[p] holds nrhs x n_p targets, right-hand side major
 *            (Ys[p][r * n_p + i]), FP64; device pointers if y_on_device
 *   nrhs     right-hand sides per problem, 1 <= nrhs <= 8
 *   lambdas  P regularisers, > 0
 *   sketch   RS_SUBSAMPLE, RS_COUNT or RS_SUBCOUNT
 *   taus     P sketch sizes (0 = the rule of rs_create), or NULL for all 0
 *   mom, opts as for rs_create (opts.cuda_stream: the stream of the whole batch);
 *            problem p draws its sketches with seed + p; opts.chunk = 0 takes the
 *            refresh period for RS_MIXED (an FP64 refresh ends every chunk) and
 *            128 slots for plain FP64 (every problem holds one chunk's S^T A)
 *   out      receives the batch; NULL on failure
 * On failure the message is rs_batch_last_error(NULL).
 */
typedef struct rs_batch rs_batch; /* opaque; owned by the library until rs_destroy_batch */
rs_status rs_create_batch(int32_t P, const rs_matrix* Xs, const double* const* Ys,
                          int32_t y_on_device, int32_t nrhs, const double* lambdas,
                          int32_t sketch, const int64_t* taus, const rs_mom* mom, uint64_t seed,
                          const rs_opts* opts, rs_batch** out);
/*
 * Solve every (problem, right-hand side) pair to relative residual tol (each
 * relative to its own ||b||), at most max_iters iterations per problem.
 *   W_out      P host pointers; W_out[p] receives nrhs x d_p weights (right-hand side
 *              major), or NULL to skip
 *   iters_out  P * nrhs iterations done per pair (pair p * nrhs + r), or NULL
 *   resid_out  P * nrhs final relative residuals (RS_MIXED: FP64 through X), or NULL
 * Returns RS_ENOTCONV if some pair did not reach tol (outputs valid), RS_ENUMERIC if
 * some pair produced NaN/Inf.
 */
rs_status rs_solve_batch(rs_batch* b, double tol, int64_t max_iters, double* const* W_out,
                         int64_t* iters_out, double* resid_out);
void rs_destroy_batch(rs_batch* b);
const char* rs_batch_last_error(const rs_batch* b);
/* setup (all problems' A, B), last solve and autotuner time in ms (the autotuner
 * runs once, in the first rs_solve_batch, outside its solve time), the CTA size of
 * the batch's iteration kernel and the number of streams its phase 1 (sketches,
 * S^T A, M^+ of every problem) is spread over, both chosen by the autotuner. Any
 * output pointer may be NULL. */
rs_status rs_batch_info(const rs_batch* b, double* setup_ms, double* solve_ms, double* tune_ms,
                        int32_t* iter_threads, int32_t* phase1_streams);
/* Fix the launch shape instead of running the autotuner: iter_threads in {128, 256,
 * 512}, phase1_streams in {1, 2, 4}; (0, 0) hands the choice back to the autotuner,
 * which then runs in the next rs_solve_batch. RS_EINVAL for other values or when the
 * iteration kernel does not fit with that CTA size. */
rs_status rs_batch_set_launch(rs_batch* b, int32_t iter_threads, int32_t phase1_streams);
/* Time the parts of a chunk: from a fresh state (tolerance 0, so that no pair
 * stops), `chunks` chunks of every problem, each part captured as its own CUDA graph
 * and timed with events. ms_parts (6 entries) receives the mean ms per chunk of:
 * the sketch plans, the sketched rows S^T A, M = S^T A S, the inverses M^+ (the four
 * parts of phase 1), the iterations, and the FP64 refresh with the end-of-chunk
 * bookkeeping. The solution state is overwritten. */
rs_status rs_batch_profile(rs_batch* b, int32_t chunks, double* ms_parts);

/*
 * Learned sketch proposal (subsample sketch of a dense context). The rows of each
 * iteration's sample are drawn without replacement from
 *   p_j = (1 - eps) softmax(s)_j + eps / m,
 * s_j the score of a 4 -> 64 -> 64 -> 1 network (ReLU; bfloat16 weights and
 * activations, FP32 accumulation) on the standardised features of row j at the
 * chunk's first iteration k0: ln A_jj, ln(1 + |r_j| / rms(r)), ln ||A[:, j]||_2,
 * ln(1 + age_j) (age_j = k0 - the last iteration whose sample held j, k0 + 1 if
 * none). The draw for iteration k: the tau rows with the largest
 * ln p_j - ln(-ln u_j), u_j = (hi32(draw(seed, k, 4, j)) + 1/2) 2^-32 (stream 4
 * of the counter-based generator; Gumbel-top-k), in increasing row order. The
 * proposal is evaluated once per chunk (opts.chunk iterations), so that the
 * chunk's sketched systems are still formed and inverted together. This replaces
 * the paper's fixed sampling probabilities (uniform, or proportional to A_jj in
 * Section 6) by predicted ones; uniform sampling stays available.
 *   w_bf16  4545 bfloat16 weights, host pointer, copied: W1 (64 x 4, row-major),
 *           b1 (64), W2 (64 x 64, row-major, W2[o, i]), b2 (64), w3 (64), b3; NULL =
 *           uniform proposal (p_j = 1 / m) drawn the same way
 *   eps     uniform share in [0, 1]; eps < 0 switches back to the plain sampler
 * RS_EUNSUPPORTED for other sketches, matrix-free contexts or m > 16384.
 */
rs_status rs_set_proposal(rs_ctx* c, const uint16_t* w_bf16, double eps);

/*
 * Training data for the learned proposal from this solver's own trajectory: from
 * the current state, up to n_iters iterations (the proposal set by rs_set_proposal
 * draws the rows), recording for every drawn row p of iteration k its features at
 * k (the layout of rs_proposal_features) and the target
 *   y_p = (1/2) ln(m max(a_p, 0) / e_k + 1e-3),  a_p = (r_C)_p delta_p,
 *   e_k = ||w_k - w*||_A^2 = (w_k - w*) . r_k,
 * where r_C . delta is the exact decrease of ||w - w*||_A^2 of a step without
 * momentum (the projection identity of Section 3). Stops early once e_k <= 0 or
 * ||r_k|| <= tol ||r_0||. Everything runs on the device; the host waits once.
 *   w_star  m doubles (host): the solution the errors are measured against
 *   Z_out   n_iters * tau * 4 floats (host), y_out n_iters * tau floats (host)
 *   n_rows  rows written
 * Needs RS_PLAIN_FP64, the subsample sketch with a proposal set, chunk = 1 and no
 * momentum (RS_EINVAL otherwise). The state advances like rs_step.
 */
rs_status rs_collect(rs_ctx* ctx, const double* w_star, int64_t n_iters, double tol, float* Z_out,
                     float* y_out, int64_t* n_rows);

/*
 * Importance-sampled subsample sketches (Section 7): with RS_SAMPLE_DIAG the tau
 * rows of iteration k are drawn without replacement in proportion to the diagonal
 * of A, p_j = A_jj / trace(A) (eq. (mSdisccolCD); for tau = 1 this is coordinate
 * descent with the probabilities of that equation, and with momentum eq. (CDmom)),
 * as the tau largest keys ln p_j + g_j with the Gumbel noise g_j of iteration k
 * (the draws of the learned proposal with its scores fixed at ln A_jj and eps = 0).
 * RS_SAMPLE_UNIFORM returns to the sketch's own uniform draws (also clears a
 * learned proposal). RS_SUBSAMPLE sketches of dense A, m <= 16384 (RS_EUNSUPPORTED
 * otherwise). Takes effect from the next rs_solve or rs_step.
 */
enum { RS_SAMPLE_UNIFORM = 0, RS_SAMPLE_DIAG = 1 };
rs_status rs_set_sampling(rs_ctx* ctx, int32_t kind);

/*
 * Accelerated sketch-and-project (Algorithm 3, Section 9) with parameters
 * 0 < mu <= 1 <= nu <= 1 / mu: beta = 1 - sqrt(mu / nu), gamma = sqrt(1 / (mu nu)),
 * alpha = 1 / (1 + sqrt(nu / mu)); three iterates w, v, z = alpha v + (1 - alpha) w
 * and the residuals r_w, r_v (r_z = alpha r_v + (1 - alpha) r_w), the sketched
 * system solved for S^T r_z. The momentum parameters of rs_create are not used while
 * it is on. mu = nu = 1 is Algorithm 1 (z = v = w). The stopping test is on
 * ||r_w|| / ||r_w^0||, the residual of the returned w (the printed listing monitors
 * r_v). mu = nu = 0 returns to Algorithm 2. Needs the persistent iteration kernel
 * (subsample, count or subcount sketch of dense A), else RS_EUNSUPPORTED; bad
 * parameters give RS_EINVAL. Takes effect from the next rs_solve or rs_step.
 */
rs_status rs_set_acceleration(rs_ctx* ctx, double mu, double nu);

/*
 * Averaged iterates (the theorem of Section 5.2, eqs. (convsublinear) and
 * (convressublinear)): with averaging on, rs_solve also keeps the running sum of
 * its iterates w^0 = 0, w^1, ..., w^t inside the iteration kernel (FP64, one add
 * per coordinate and iteration), and rs_get_average returns their mean
 * wbar^t = (w^0 + ... + w^t) / (t + 1) of the last rs_solve (the paper writes the
 * sum over t + 1 iterates with a factor 1 / t; the mean is read here). For RS_DUAL
 * the result is X^T of the mean of the dual iterates, like w of rs_solve.
 *   rs_set_averaging  on = 1 / 0; needs the persistent iteration kernel (subsample,
 *                     count or subcount sketch of dense A): RS_EUNSUPPORTED otherwise.
 *                     Takes effect from the next rs_solve.
 *   rs_get_average    w_out: d doubles, caller-owned, device memory if w_on_device;
 *                     RS_EINVAL when averaging is off.
 */
rs_status rs_set_averaging(rs_ctx* ctx, int32_t on);
rs_status rs_get_average(rs_ctx* ctx, double* w_out, int32_t w_on_device);
/* The m x 4 standardised feature rows (FP32, row-major, host pointer) at the
 * context's current state, as the proposal would see them at a chunk start. */
rs_status rs_proposal_features(rs_ctx* c, float* Z_out);

/*
 * Training the proposal's network: FP32 master weights, Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8, bias-corrected), and the bfloat16 copy that the forward uses.
 * The loss is mean((s - y)^2) / 2 over the rows; the forward rounds weights and
 * hidden activations to bfloat16 and the gradient passes those roundings
 * straight through. Z (n x 4 FP32, row-major) and y (n FP32) are device
 * pointers; everything runs on `stream` (NULL = default stream).
 */
typedef struct rs_mlp rs_mlp; /* opaque; owned by the library until rs_mlp_destroy */
rs_status rs_mlp_create(const float* theta0 /* host, 4545 */, int32_t device, void* stream,
                        rs_mlp** out);
/* gradient (host, 4545; NULL to skip) and loss at the current weights */
rs_status rs_mlp_grad(rs_mlp* h, const float* Z, const float* y, int64_t n, float* grad_out,
                      double* loss_out);
/* one Adam step on the rows; the loss before the step (NULL to skip) */
rs_status rs_mlp_step(rs_mlp* h, const float* Z, const float* y, int64_t n, double lr,
                      double* loss_out);
/* scores of n feature rows into s_out (device, n FP32), asynchronous */
rs_status rs_mlp_scores(rs_mlp* h, const float* Z, int64_t n, float* s_out);
/* FP32 master weights and/or their bfloat16 copy (host pointers, 4545 each) */
rs_status rs_mlp_get(rs_mlp* h, float* theta_out, uint16_t* bf16_out);
void rs_mlp_destroy(rs_mlp* h);
const char* rs_mlp_last_error(const rs_mlp* h);

#ifdef __cplusplus
}
#endif
#endif /* RIDGESKETCH_H */

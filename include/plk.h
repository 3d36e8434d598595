/*
 * plk.h -- C ABI of the B300 profile-likelihood library (libplk.so).
 *
 * The library evaluates the profile log-likelihood l_p(omega, lambda) of the
 * Box-Cox linear geostatistical model with anisotropic Matern correlation
 * (Xu & Brown, arXiv 2305.04318) at many correlation-parameter points omega and
 * Box-Cox parameters lambda:
 *   model        Y' ~ MVN(X beta, sigma^2 V), V = R(omega) + nu^2 I      (Section 2, eq. 1)
 *   correlation  rho = 2^{1-kappa}/Gamma(kappa) u^kappa K_kappa(u),
 *                u = sqrt(8 kappa) d(x), d = ||diag(1/phi_X, 1/phi_Y) Rot(phi_A) x||
 *                                                                     (Section 2, eq. matern)
 *   statistics   log|V|, log|X'V^-1X|, (y',X)'V^-1(y',X), ssqBetahat,
 *                ssqResidual                                          (Section 3.3, Table 1)
 *   closed form  beta-hat, sigma-hat^2 and
 *                -2 l_p = n log(RSS/n) + log|V| - 2(lambda-1) sum log y + n log(2 pi) + n
 *                                                                     (eqs. betahat, 4, profile)
 *   REML         -2 l*_p = (n-p) log(RSS/(n-p)) + log|V| + log|X'V^-1X|
 *                          - 2(lambda-1) sum log y + n log(2 pi) + n - p   (Appendix, eq. remlpro)
 *   profile CI   {theta : l_p(theta) >= max l_p - chi2_1(level)/2}    (Section 2.2, eq. likelihood)
 *
 * Parameter point layout (one row of 5 doubles, "natural" parameters):
 *   [0] phi_X   range, > 0
 *   [1] kappa   Matern shape, > 0
 *   [2] nu^2    nugget ratio tau^2/sigma^2, >= 0
 *   [3] phi_R   anisotropy ratio phi_X/phi_Y, > 0 (phi_Y = phi_X / phi_R)
 *   [4] phi_A   anisotropy angle in radians (rotation matrix as printed in eq. matern)
 *
 * Conventions for every call:
 *   - Returns a plk_status; PLK_OK on success.  On failure nothing is written to
 *     caller output buffers and plk_last_error() describes the cause.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *     memory on the context's / call's device.  Row-major layouts throughout.
 *   - The caller owns every buffer it passes; the library copies inputs it keeps.
 *   - A numerical failure at one omega point (V or X'V^-1X not positive definite,
 *     or a non-positive residual sum of squares) is not a call failure: that
 *     point's status is set and its outputs are NaN.
 *   - No call falls back to a CPU implementation.  A missing or unusable GPU is
 *     PLK_E_CUDA.
 */
#ifndef PLK_H
#define PLK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PLK_OK = 0,
    PLK_E_INVALID = 1,   /* bad argument: sizes, NULL required pointer, y <= 0, non-finite, ... */
    PLK_E_NOMEM = 2,     /* workspace / HBM budget too small for even one omega point */
    PLK_E_NOT_READY = 3, /* poll: the job has not finished within the timeout */
    PLK_E_TIMEOUT = 4,   /* a bounded device-side wait gave up */
    PLK_E_CUDA = 5,      /* a CUDA runtime or launch error */
    PLK_E_CANCELLED = 6  /* job cancelled */
} plk_status;

/* Per-point status codes written to point_status[]. */
#define PLK_POINT_OK 0
#define PLK_POINT_NOT_PD 1       /* V (or X'V^-1X) not positive definite in the working precision */
#define PLK_POINT_BAD_PARAM 2    /* parameter row outside its domain (phi_X<=0, kappa<=0, ...) */
#define PLK_POINT_RSS_NONPOS 3   /* residual sum of squares <= 0 */
#define PLK_POINT_RETRIED 16     /* flag bit: mixed mode re-evaluated this point with the 7-slice
                                    (~48-bit) split because the 5-slice error bound was too large */
#define PLK_POINT_FP64 32        /* flag bit: mixed mode re-evaluated this point in FP64 because the
                                    7-slice error bound was still too large */

typedef enum {
    PLK_FP64 = 0,  /* every step in FP64 arithmetic */
    PLK_MIXED = 1  /* FP64 build / diagonal blocks / log-det / quadratic forms; trailing
                      updates and TRSM bulk as exact split-bf16 products on the tensor cores */
} plk_precision;

typedef struct {
    int32_t precision;  /* plk_precision */
    int32_t reml;       /* 0: ML profile (eq. profile); 1: REML profile (eq. remlpro) */
    int32_t batch;      /* omega points per device batch, <= 65535; 0 = library default */
    int32_t flags;      /* PLK_FLAG_* bits */
} plk_options;

/* flags: bracket every kernel launch with CUDA events on its stream and
 * accumulate the elapsed time per kernel class (read with plk_kernel_timing). */
#define PLK_FLAG_KERNEL_TIMING 1
/* flags: PLK_MIXED without the 7-slice re-evaluation of points whose error bound
 * exceeds the tolerance (for measuring the 5-slice error itself). */
#define PLK_FLAG_NO_RETRY 2
/* flags: PLK_MIXED without the FP64 re-evaluation tier (keeps the 7-slice result;
 * for measuring the 7-slice error itself). */
#define PLK_FLAG_NO_FP64_TIER 4
/* flags: launch each batch's kernel sequence as one CUDA graph (PLK_FP64: the
 * whole batch; PLK_MIXED: the whole batch too -- the 5-slice pass, the 7-slice
 * tier, whose points are compacted on the device and whose kernels take their
 * live count from device memory, and the FP64 tier as the body of a
 * conditional node that runs only when its device-side count is positive).
 * On the legacy default stream, which cannot be captured, the launches stay
 * eager.  The sequence is captured from
 * the stream with the same launch code and replayed; between batches of the
 * same shape the executable graph is only updated.  Results are identical to
 * the eager launches.  Ignored together with PLK_FLAG_KERNEL_TIMING. */
#define PLK_FLAG_GRAPH 8
/* flags: PLK_MIXED, run the 5-slice pass to the end on every point.  By default
 * a point stops in that pass once the partial sum of its error bound (which
 * only grows with further pivots) exceeds the tolerance, or its factorisation
 * fails: it is re-evaluated with 7 slices in either case, so the results are
 * identical with and without this flag (it exists for that check and for
 * timing the full pass).  PLK_FLAG_NO_RETRY implies it. */
#define PLK_FLAG_FULL_FIRST_PASS 16
/* flags: keep small datasets on the tiled path.  By default a dataset with
 * n + M + p <= 224 is evaluated by one fused kernel per batch: one thread
 * block per point builds the bordered matrix in shared memory, factors it and
 * leaves the cross-products for the closed form -- in FP64 for PLK_FP64; in
 * double-float FP32 arithmetic for PLK_MIXED, where a point whose
 * a-posteriori bound 2^-36 (1 + nu^2) sum_j 1/d_j exceeds the mixed tolerance
 * (plk_set_mixed_tolerance; or whose
 * factorisation fails) is evaluated again in FP64 (status bits RETRIED and
 * FP64, err_bound 0).  This flag selects the tiled path instead (for
 * comparisons). */
#define PLK_FLAG_NO_FUSED 32
/* flags: PLK_MIXED, batches of >= 256 points: re-evaluate the points each
 * part of the 5-slice pass (about 296 points) sends to the 7-slice tier on a
 * low-priority stream as soon as that part is done, beside the later parts,
 * instead of once after the whole pass (the default).  Results are identical
 * either way.  Measured slower at n = 4000 (1375 vs 1426 evals/s): the
 * re-evaluation's kernels hold SMs that the pass's persistent trailing update
 * then waits for. */
#define PLK_FLAG_PIPELINED_RETRY 64

/* ------------------------------------------------------------------------ */
/* Stateless device-pointer evaluation (one dataset, K points)               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;               /* sites, n > p */
    int32_t p;               /* covariates, 1 <= p <= 16 */
    int32_t M;               /* lambda values, M >= 1, M + p <= 64 */
    const double *coords;    /* device, n x 2 site coordinates */
    const double *y;         /* device, n observations, all > 0 */
    const double *X;         /* device, n x p design matrix */
    const double *lambdas;   /* device, M Box-Cox parameters */
    int64_t K;               /* number of parameter points, >= 0 */
    const double *params;    /* device, K x 5 parameter points (layout above) */
    /* outputs, device, any may be NULL */
    double *logL;            /* K x M  l_p(omega_k, lambda_m) (or l*_p if reml) */
    double *sigma2;          /* K x M  sigma-hat^2 (RSS/n, or RSS/(n-p) if reml) */
    double *beta;            /* K x M x p beta-hat */
    double *logdet;          /* K x 2  [log|V|, log|X'V^-1X|] */
    int32_t *status;         /* K      PLK_POINT_* codes */
    double *err_bound;       /* K      PLK_MIXED: a-posteriori bound on |Delta l_p| of the split-product
                                       factorisation that produced the result (0 for points
                                       re-evaluated in FP64); PLK_FP64: 0 */
    double *ssq_yx;          /* K x (M+p) x (M+p)  (y',X)^T V^-1 (y',X), the ssqYX of Table 1
                                       (Section 3.3 Step 3 item 4): symmetric, row-major per
                                       point, the M columns y'(lambda_m) first, then X; NaN
                                       where V or X^T V^-1 X is not positive definite or the
                                       parameter row is invalid */
} plk_eval_args;

/* Bytes of device workspace plk_eval_device needs to process `batch` points of
 * a dataset with n sites, p covariates and M lambdas in the given precision.
 * Returns 0 for invalid sizes. */
size_t plk_eval_workspace_bytes(int64_t n, int32_t p, int32_t M, int32_t batch,
                                int32_t precision);

/* Diagnostics of a library built with -DPLK_PIPE_COUNTERS (libplk_counters.so,
 * paper_2305_04318_b300/build.py): cycles the 5-slice trailing update's roles
 * spent waiting, per launch mode (0 the trailing triangle, 1 a tile column, 2
 * the right-hand-side row), summed over its thread blocks since the last
 * reset.  out (host, 27 values): [mode * 9 + k], k = 0 cycles of the blocks'
 * work loops, 1 items, 2 MMA issue waiting for a free accumulator set, 3 ...
 * for a B operand buffer, 4 ... for an A stage, 5 epilogue waiting for the
 * item's MMAs, 6 ... for its C half tile, 7 ... for the previous stores to
 * read the C buffer, 8 epilogue update.  reset != 0 zeroes the counters after
 * reading.  Errors: PLK_E_INVALID (NULL out, or a library built without the
 * counters), PLK_E_CUDA. */
plk_status plk_pipe_counters(uint64_t *out, int32_t reset);

/* Tolerance of the PLK_MIXED retry rule: a point whose a-posteriori bound on
 * |Delta l_p| exceeds it is evaluated again (5 slices -> 7 slices -> FP64; for
 * small datasets double-float -> FP64).  Process-wide, read when a batch is
 * enqueued; default 1e-3 (the mixed mode's accuracy target in absolute log-L
 * units).  A smaller value sends more points to the slower tiers.
 * Errors: PLK_E_INVALID unless 0 < tol <= 1 (the setting is unchanged). */
plk_status plk_set_mixed_tolerance(double tol);
double plk_get_mixed_tolerance(void);

/* Evaluate all K points of `args` on `stream` (a cudaStream_t, 0 = legacy
 * default stream), in batches of opts->batch points, using only the caller's
 * workspace (device, `workspace_bytes` >= plk_eval_workspace_bytes(...), 256-byte
 * aligned).  Allocates nothing.  Asynchronous: returns after enqueueing; outputs
 * are valid once the stream reaches this point.  Errors: PLK_E_INVALID (sizes,
 * NULL inputs), PLK_E_NOMEM (workspace too small for opts->batch), PLK_E_CUDA
 * (launch failure). */
plk_status plk_eval_device(const plk_eval_args *args, const plk_options *opts, void *workspace,
                           size_t workspace_bytes, void *stream);

/* Covariance matrices V(omega_k) = R(omega_k) + nu_k^2 I of eq. (matern)
 * (Section 2; the first item of Step 3 in Section 3.3), as the evaluation
 * builds them, written out densely.
 *   coords    device, n x 2 site coordinates (n >= 2)
 *   params    device, K x 5 parameter points (layout above), 1 <= K <= 65535
 *   mode      0: FP64 entries (the PLK_FP64 path's build);
 *             1: double-float entries evaluated in FP32 pair arithmetic (the
 *                first, 5-slice pass of the PLK_MIXED path);
 *             2: double-float entries evaluated in FP64 (the 7-slice tier of
 *                the PLK_MIXED path); modes 1 and 2 return hi + lo as doubles
 *   V         device, K x n x n row-major, both triangles (caller-owned); rows
 *             of a point whose parameters are invalid hold the build's fill
 *   workspace device, >= plk_eval_workspace_bytes(n, 1, 1, K, PLK_FP64) bytes,
 *             256-byte aligned (caller-owned scratch)
 * Allocates nothing; asynchronous on `stream`.  Errors: PLK_E_INVALID (sizes,
 * NULL pointers, mode, alignment), PLK_E_NOMEM (workspace too small),
 * PLK_E_CUDA (launch failure). */
plk_status plk_build_covariance_device(const double *coords, int64_t n, const double *params, int64_t K,
                                       int32_t mode, double *V, void *workspace, size_t workspace_bytes,
                                       void *stream);

/* Evaluation without any device allocation (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory when they evaluate -- for
 * example a plugin whose host application owns the entire device-memory
 * budget, or a latency-critical loop that must not call cudaMalloc/cudaFree
 * because those calls can stall or synchronize other work on the device.
 * Same computation and outputs as plk_eval_device in PLK_FP64 (ML if reml == 0,
 * REML otherwise); the scratch it needs lives in one device array of
 * PLK_STATIC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.  The caller passes inputs and outputs
 * (device pointers, as for plk_eval_device) and a stream.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any
 *     stream capture.
 *   - Every call on a device shares the same array.  Calls that overlap on the
 *     GPU (other streams, other host threads) race on it and give wrong
 *     results; serialize them.  Nothing needs to start at zero: each call
 *     writes every scratch byte before it reads it, so contents left by the
 *     previous call do not matter.
 *   - Points are processed in batches as large as fit in the array.  Sizes for
 *     which even one point does not fit (n above about 3840) are rejected with
 *     PLK_E_NOMEM before any work is queued; use plk_eval_device then.
 *   - Allocates nothing and calls no allocating routine.  Asynchronous on
 *     `stream` like plk_eval_device. */
#define PLK_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
plk_status plk_eval_device_static(const plk_eval_args *args, int32_t reml, void *stream);

/* ------------------------------------------------------------------------ */
/* Context API: device-resident datasets, asynchronous jobs                  */
/* ------------------------------------------------------------------------ */

typedef struct plk_ctx plk_ctx;
typedef int64_t plk_dataset;
typedef int64_t plk_job;

/* Create a context on CUDA device `device`.  `arena` (device memory owned by the
 * caller, e.g. a PyTorch tensor) of `arena_bytes` is where the context places
 * datasets and job workspaces; when arena is NULL the context allocates
 * `arena_bytes` itself with cudaMalloc at creation and frees it at destroy.
 * All admission of work is bounded by this arena (the HBM budget).
 * `streams` (cudaStream_t handles, may be NULL) / `n_streams` are the streams
 * the scheduler launches on; when NULL the context creates `n_streams` (>= 1)
 * non-blocking streams of its own. */
plk_status plk_create(plk_ctx **out, int device, void *arena, size_t arena_bytes,
                      void *const *streams, int n_streams);

/* Copy a dataset (host pointers) to the device: coords n x 2, y n (> 0), X n x p.
 * Validates: n > p >= 1, p <= 16, finite values, y > 0. */
plk_status plk_create_dataset(plk_ctx *ctx, const double *coords, const double *y,
                              const double *X, int64_t n, int32_t p, plk_dataset *out);

/* Submit a profile job: K parameter points (host, K x 5) x M lambdas (host).
 * The inputs are copied before return; the job runs asynchronously and
 * interleaves with other jobs as arena space and streams free up.
 * PLK_E_NOMEM if even one point of this dataset cannot fit in the arena. */
plk_status plk_submit_profile(plk_ctx *ctx, plk_dataset ds, const double *param_grid, int64_t K,
                              const double *lambda_grid, int32_t M, const plk_options *opts,
                              plk_job *out);

/* Wait up to timeout_ms (0 = do not wait, < 0 = wait forever) for `job`; on
 * completion copy its results into the caller's host buffers (any may be NULL;
 * layouts as in plk_eval_args) and forget the job.  PLK_E_NOT_READY if still
 * running.  Timing of the job (host clock, seconds since context creation) is
 * returned in t_submit/t_start/t_done when non-NULL. */
plk_status plk_poll(plk_ctx *ctx, plk_job job, int32_t timeout_ms, double *logL, double *sigma2,
                    double *beta, double *logdet, int32_t *point_status, double *t_submit,
                    double *t_start, double *t_done);

/* Release a dataset's device memory (after its jobs have completed). */
plk_status plk_release_dataset(plk_ctx *ctx, plk_dataset ds);

/* Arena statistics: bytes in use now and the high-water mark. */
plk_status plk_memory_stats(plk_ctx *ctx, size_t *in_use, size_t *high_water);

/* Wait for all jobs, free everything the context owns. */
plk_status plk_destroy(plk_ctx *ctx);

/* Cancel a job (the paper has no counterpart: its back end runs a fixed grid
 * to the end).  Batches of the job not yet launched are dropped; batches
 * already running on the device finish (kernels are not interrupted) and
 * their results are discarded.  Once nothing of the job is running, plk_poll
 * returns PLK_E_CANCELLED for it and forgets it.  Cancelling a job that has
 * already completed has no effect: plk_poll still returns its results.
 * PLK_E_INVALID for an unknown job. */
plk_status plk_cancel(plk_ctx *ctx, plk_job job);

/* Which job's next batch a free scheduler stream takes (no counterpart in
 * the paper, whose back end runs one grid at a time):
 *   PLK_SCHED_FIFO           the oldest job with work left (the default;
 *                            serving: the earliest request is served first);
 *   PLK_SCHED_LARGEST_FIRST  the job on the largest dataset (cost per point
 *                            ~ n^3), the oldest among equals (many jobs
 *                            submitted together: the small ones fill the end
 *                            instead of a large one running alone).
 * Results do not depend on the policy.  PLK_E_INVALID for an unknown policy. */
#define PLK_SCHED_FIFO 0
#define PLK_SCHED_LARGEST_FIRST 1
plk_status plk_set_schedule_policy(plk_ctx *ctx, int32_t policy);

/* Per-job metrics as JSON lines (no counterpart in the paper).  From this call
 * on, every job that ends (completed, failed or cancelled) appends one line to
 * the file at `path` (opened for appending; NULL stops logging): job and
 * dataset ids, n, p, M, K, precision, reml, points per batch, number of
 * batches ("items"), outcome, host times t_submit / t_start / t_done (seconds
 * since context creation), queue wait (t_start - t_submit), run time, the
 * summed and the p50 / p99 wall time of its batches, evaluations per second,
 * the counts of points not ok / re-evaluated with 7 slices / in FP64, and the
 * arena's bytes in use and high-water mark.  PLK_E_INVALID if the file cannot
 * be opened. */
plk_status plk_set_metrics_log(plk_ctx *ctx, const char *path);

/* Host-side fault hooks, for tests of failure handling without a GPU fault
 * (no counterpart in the paper).  The next `count` events of the given kind
 * fail (count 0 clears the hook):
 *   PLK_FAULT_ARENA_ALLOC      a batch's workspace allocation in the arena
 *                              fails as if the arena were full: the scheduler
 *                              halves the batch, then waits and retries, so
 *                              the job completes with the same results;
 *   PLK_FAULT_BATCH            a batch fails before it is launched, as a failed
 *                              launch would: its job stops launching and
 *                              plk_poll returns PLK_E_CUDA with the message
 *                              "injected batch failure (fault hook)"; other
 *                              jobs are unaffected;
 *   PLK_FAULT_DROP_COMPLETION  the wake-up of threads waiting in plk_poll for
 *                              a finished job is not sent: plk_poll still sees
 *                              the job done within 50 ms (it re-checks).
 * Nothing here touches the GPU.  PLK_E_INVALID for an unknown kind or a
 * negative count. */
#define PLK_FAULT_ARENA_ALLOC 1
#define PLK_FAULT_BATCH 2
#define PLK_FAULT_DROP_COMPLETION 3
plk_status plk_inject_fault(plk_ctx *ctx, int32_t kind, int32_t count);

/* Evaluator of a batch of points on the host: for the `count` parameter rows
 * `params` (count x 5) of the dataset (coords n x 2, y n, X n x p; host
 * memory) and the M lambdas, write logL, sigma2 (count x M), beta
 * (count x M x p), logdet (count x 2) and status (count), layouts as in
 * plk_eval_args.  Returns 0 on success; anything else fails the batch. */
typedef int (*plk_host_eval_fn)(void *user, int64_t n, int32_t p, const double *coords, const double *y,
                                const double *X, const double *params, int64_t count, const double *lambdas,
                                int32_t M, double *logL, double *sigma2, double *beta, double *logdet,
                                int32_t *status);

/* A context whose scheduler runs every batch on the host through `fn` (with
 * `user`) on n_workers worker threads (1 .. 64), with an arena of arena_bytes
 * of host memory, instead of launching the library's kernels on a GPU (no
 * counterpart in the paper).  It exists to test the scheduler itself --
 * admission, continuous batching, cancellation, the fault hooks and the
 * metrics log -- on machines without a GPU, with any evaluator (the library's
 * tests pass a CPU reference implementation).  It is never chosen
 * implicitly: the GPU calls never fall back to it.  Every context call works
 * on it except plk_autotune (PLK_E_INVALID).  Errors: PLK_E_INVALID,
 * PLK_E_NOMEM (host arena). */
plk_status plk_create_with_evaluator(plk_ctx **out, size_t arena_bytes, int n_workers, plk_host_eval_fn fn,
                                     void *user);

/* Autotuner of the batch schedule (the paper fixes its batch, NparamPerIter,
 * by hand for its unnamed GPU; Section 4).  Times this context's scheduler on a
 * synthetic dataset of n sites with p covariates and M lambdas: for each
 * candidate batch size b (NULL / 0 candidates: 32, 64, 148, 296, 592), one
 * job of 2 b x (number of streams) points from submit to host results; keeps the
 * fastest b for n's half-octave bucket and precision.  Later jobs submitted
 * with opts->batch == 0 on datasets whose n falls in that bucket or a
 * neighbouring one use it.  Candidates whose batches do not fit in the free
 * arena are skipped.  Blocking; runs the context's own kernels (its datasets
 * and jobs stay valid).  The tile size is fixed at 128 by the tensor-core
 * shapes; the batch is what is tuned.  Outputs (may be NULL): the chosen
 * batch and its points per second.  Errors: PLK_E_INVALID, PLK_E_NOMEM (no
 * candidate fits), PLK_E_CUDA. */
plk_status plk_autotune(plk_ctx *ctx, int64_t n, int32_t p, int32_t M, int32_t precision,
                        const int32_t *candidates, int32_t n_candidates, int32_t *best_batch,
                        double *best_rate);

/* Batch size the scheduler uses for a job of K points on a dataset of n sites
 * in `precision` when opts->batch == 0; *tuned (may be NULL) = 1 if it comes
 * from plk_autotune, 0 if it is the library default. */
plk_status plk_scheduled_batch(plk_ctx *ctx, int64_t n, int32_t precision, int64_t K, int32_t *batch,
                               int32_t *tuned);

/* ------------------------------------------------------------------------ */
/* Steps 1 and 2 of the method (Sections 3.1-3.2): the maximum-likelihood     */
/* estimate and the representative parameter points                          */
/* ------------------------------------------------------------------------ */

/* Internal parameters (Section 3.2), one row of 5 doubles:
 *   [0] gamma_1 = log phi_X + log phi_Y            (sumLogRange)
 *   [1] kappa~  = log kappa, or 1/sqrt(kappa) when the fitted kappa >= 4
 *   [2] nu      = sqrt(nu^2)
 *   [3] gamma_2 = sqrt(phi_X/phi_Y - 1) cos(2 phi_A) (aniso1)
 *   [4] gamma_3 = sqrt(phi_X/phi_Y - 1) sin(2 phi_A) (aniso2)
 * (natural -> internal: plk_internal_params_device.)  Host: natural rows of K
 * internal rows; phi_R = 1 + gamma_2^2 + gamma_3^2 >= 1, phi_A =
 * atan2(gamma_3, gamma_2)/2 in [0, pi), nu^2 = nu^2.  Errors: PLK_E_INVALID. */
plk_status plk_natural_params(const double *internal, int64_t K, int32_t kappa_hat_large, double *out);

/* chi^2 quantile: x with P(chi^2_dof <= x) = p (host; NaN for
 * dof < 1 or p outside (0, 1)).  The contour levels of Section 3.2. */
double plk_chi2_quantile(int32_t dof, double p);

/* The numerical-Hessian stencil of Section 3.2 around `center_internal` (host,
 * 5 doubles) in the free internal coordinates (all five, or all but kappa~
 * when kappa_fixed): the centre, +-delta e_i, and +-delta e_i +-delta e_j for
 * every pair i < j in the order (+,+), (+,-), (-,+), (-,-): S = 2 d^2 + 1 rows
 * (51 for d = 5, 33 for d = 4) of internal parameters written to `out`
 * (host, S x 5); *S_out = S.  Errors: PLK_E_INVALID. */
plk_status plk_hessian_stencil(const double *center_internal, int32_t kappa_fixed, double delta, double *out,
                               int32_t *S_out);

/* Hessian H (d x d) and gradient (d) of L(omega') = max over lambda of l_p,
 * from l_p at the stencil rows (host, S x 3: lambda-hat - dl, lambda-hat,
 * lambda-hat + dl per row).  Per row, L is the maximum of the parabola through
 * the three values over lambda-hat + t dl, |t| <= tmax (the largest of the
 * three when the parabola is not concave; NaN if any is NaN); then central
 * differences: H_ii = (L(+i) - 2 L(0) + L(-i))/delta^2, H_ij = (L(++) - L(+-)
 * - L(-+) + L(--))/(4 delta^2), g_i = (L(+i) - L(-i))/(2 delta).  Optional
 * outputs: the profiled L (S) and the offsets t (S).  Host; PLK_E_INVALID. */
plk_status plk_hessian_from_stencil(int32_t kappa_fixed, double delta, const double *logL3, double tmax, double *H,
                                   double *grad, double *L_profiled, double *t_lambda);

/* Eigen-decomposition -H = E diag(D) E^T (host, d <= 5; E's columns the
 * eigenvectors) with the fix-up of Section 3.2: negative eigenvalues replaced
 * by their absolute values; if the largest exceeds 100, eigenvalues below 0.1
 * become 0.1; numerically zero ones (below 1e-8 max(1, largest)) or non-finite
 * ones become 0.1.  PLK_E_INVALID. */
plk_status plk_fix_hessian(int32_t d, const double *H, double *E, double *D);

/* n points on the unit sphere in R^d spread by a stochastic maximin optimiser
 * (maximises the smallest pairwise distance, Section 3.2), seeded; `rounds`
 * passes over the points.  Host, x: n x d; *min_distance (may be NULL) the
 * smallest pairwise distance reached.  PLK_E_INVALID. */
plk_status plk_sphere_points(int32_t d, int32_t n, uint64_t seed, int32_t rounds, double *x,
                             double *min_distance);

/* Likelihood evaluator for the two steps below: l_p (K x M, row-major) at K
 * natural parameter rows (K x 5) and M lambdas; returns 0 on success, else a
 * plk_status.  plk_fit_mle / plk_quadratic_cloud use the library's own GPU
 * evaluation through a context; the _cb forms take any evaluator. */
typedef int32_t (*plk_eval_fn)(void *user, const double *params, int64_t K, const double *lambdas, int32_t M,
                               double *logL);

typedef struct {
    int32_t precision;    /* plk_precision of the evaluations (context forms) */
    int32_t reml;         /* 1: maximise the REML profile likelihood (eq. remlpro; context forms) */
    int32_t kappa_fixed;  /* 1: kappa held at `kappa` (the constrained fits of Section 3.1) */
    double kappa;
    double delta;         /* stencil step in internal coordinates; <= 0: 0.05 */
    double delta_lambda;  /* lambda step; <= 0: 0.05 */
    int32_t max_iter;     /* <= 0: 60 */
    double tol;           /* stop when an iteration gains less than tol in l_p; <= 0: 1e-7 */
} plk_fit_options;

/* Step 1 (Section 3.1): maximise l_p(omega, lambda) from (omega0, lambda0).
 * Batched Newton iteration in the internal parameters: each iteration
 * evaluates the Hessian stencil at three lambdas (one batch), takes the Newton
 * direction of the lambda-profiled likelihood with the eigenvalues of -H made
 * positive (trust radius 1 in internal units), and evaluates a batch of step
 * lengths at the lambda of the centre's parabola; the best evaluated point of
 * both batches becomes the next iterate (kappa projected onto [0.1, 20], the
 * shapes the method explores).  When an iteration
 * gains less than opts->tol both finite-difference steps shrink by 4 (at most
 * twice); it stops when that no longer helps or after opts->max_iter.  Outputs (host): omega_hat (5, natural), lambda_hat,
 * logL_hat (l_p evaluated at them, may be NULL), iterations (may be NULL).
 * Errors: PLK_E_INVALID (start outside the domain or l_p not finite there),
 * evaluation errors. */
plk_status plk_fit_mle(plk_ctx *ctx, plk_dataset ds, const double *omega0, double lambda0,
                       const plk_fit_options *opts, double *omega_hat, double *lambda_hat, double *logL_hat,
                       int32_t *iterations);
plk_status plk_fit_mle_cb(plk_eval_fn fn, void *user, const double *omega0, double lambda0,
                          const plk_fit_options *opts, double *omega_hat, double *lambda_hat, double *logL_hat,
                          int32_t *iterations);

typedef struct {
    int32_t precision;          /* plk_precision of the stencil evaluations (context form) */
    int32_t reml;               /* 1: the REML profile likelihood (eq. remlpro; context form) */
    int32_t kappa_fixed;        /* 1: 4-D cloud with kappa held at omega_hat's kappa */
    int32_t n_sphere;           /* points per contour level; <= 0: 726 (5-D) or 120 (4-D) */
    int32_t n_levels;           /* contour levels (with level_probs) */
    const double *level_probs;  /* chi^2_d probabilities of the levels; NULL: 0.05, 0.15, ..., 0.95, 0.99 */
    int32_t n_lambda;           /* lambda grid size (0: none written) */
    double delta;               /* Hessian stencil step; <= 0: 0.05 */
    double delta_lambda;        /* <= 0: 0.05 */
    uint64_t seed;              /* sphere points and the nugget repair */
    int32_t sphere_rounds;      /* <= 0: 200 */
} plk_cloud_options;

/* Step 2 (Section 3.2): representative points around (omega_hat, lambda_hat).
 * Evaluates the Hessian stencil (one batch of S x 3 evaluations; with steps of
 * 1/4, at most twice more, while a stencil value is not finite), fixes the
 * eigenvalues of -H, spreads n_sphere maximin points on the unit sphere and
 * maps them to every contour level: x' = omega'-hat + sqrt(c_l) E D^{-1/2} E^T x
 * with c_l the chi^2_d quantile of the level, in internal coordinates, then to
 * natural rows.  A point whose nu comes out negative (a negative nugget) gets
 * nu^2 = 0 or, alternately, a uniform draw on (0, 2).  The lambda grid has
 * n_lambda values evenly spaced between the 0.01 and 0.99 quantiles of the
 * normal approximation N(lambda_hat, -1/l''(lambda)) at the centre (sd 0.5 if
 * l'' >= 0).  Outputs (host): params_out (capacity x 5; *K_out = levels x
 * n_sphere rows; with params_out NULL only *K_out is set), lambdas_out
 * (n_lambda), hessian_out (d x d), eig_out (d, the fixed eigenvalues of -H);
 * any but K_out may be NULL.  Errors: PLK_E_INVALID, PLK_E_NOMEM (capacity
 * below K), evaluation errors. */
plk_status plk_quadratic_cloud(plk_ctx *ctx, plk_dataset ds, const double *omega_hat, double lambda_hat,
                               const plk_cloud_options *opts, double *params_out, int64_t capacity, int64_t *K_out,
                               double *lambdas_out, double *hessian_out, double *eig_out);
plk_status plk_quadratic_cloud_cb(plk_eval_fn fn, void *user, const double *omega_hat, double lambda_hat,
                                  const plk_cloud_options *opts, double *params_out, int64_t capacity,
                                  int64_t *K_out, double *lambdas_out, double *hessian_out, double *eig_out);

/* Failure-detection self-test (the paper has no counterpart).  Every wait of
 * the tensor-core kernels on an mbarrier is bounded: when it gives up, the
 * kernel sets a device error flag, drains its own work and returns, and the
 * host call reports PLK_E_TIMEOUT with the device still usable.  This call
 * runs one block that waits, with the same bounded wait limited to max_iter
 * tries (1 .. 1e6; each try takes well under a microsecond), on a barrier that
 * nothing completes, so it always gives up: the expected result is
 * PLK_E_TIMEOUT.  Blocking on `stream`; concurrent calls share one device
 * flag (run them one at a time).  PLK_E_INVALID for max_iter outside its
 * range, PLK_E_CUDA for a CUDA error. */
plk_status plk_selftest_bounded_wait(int32_t max_iter, void *stream);

/* Self-test of the double-float exponential that the mixed path's first pass
 * uses in its Matern table (the paper has no counterpart: it evaluates in FP64
 * throughout).  For i < count: yh[i] + yl[i] = exp(xh[i] + xl[i]), computed
 * the way the table does it (k ln 2 + r with a three-part ln 2, a degree-9
 * Taylor polynomial of e^(r/4), two double-float squarings, then 2^k).  Its
 * relative error is ~2^-45 for arguments >= -50; below -86 the result is 0,
 * above 86 infinity.  All four arrays are device memory of `count` floats
 * (count <= 2^31), caller-owned; asynchronous on `stream`.  PLK_E_INVALID for
 * a bad count or a NULL pointer, PLK_E_CUDA for a launch error. */
plk_status plk_selftest_df_exp(const float *xh, const float *xl, float *yh, float *yl, int64_t count,
                               void *stream);

/* Message describing the last error of the calling thread ("" if none). */
const char *plk_last_error(void);

/* ------------------------------------------------------------------------ */
/* Profile reduction and likelihood CI (Section 3.6, eq. likelihood)          */
/* ------------------------------------------------------------------------ */

/* prof[g] = max over the SM consecutive values vals[g*SM .. (g+1)*SM) that are
 * not NaN (NaN if all are NaN), for g < G.  Device pointers, runs on `stream`. */
plk_status plk_profile_max_device(const double *vals, int64_t G, int64_t SM, double *prof,
                                  void *stream);

/* Likelihood-based CI from a 1-D profile on an ascending grid (device
 * pointers; results written to the device array out[4] = {lo, hi, argmax,
 * censored}).  argmax is the lowest index among ties; threshold = max -
 * chi2_1(level)/2; each endpoint interpolates linearly between the first finite
 * grid point strictly below the threshold (walking outward from the argmax) and
 * the finite point just inside it; a side that never drops below is the grid
 * edge with censored bit 1 (lower) / 2 (upper); out = NaN if no value is
 * finite.  level in (0, 1). */
plk_status plk_profile_ci_device(const double *grid, const double *prof, int64_t G, double level,
                                 double *out, void *stream);

/* The same likelihood CI (Section 2.2, eq. likelihood) for a caller holding the
 * grid and the profile in host memory: grid and profile_logL host arrays of G
 * values; outputs (host) lo, hi, argmax (the grid value at the maximum) and
 * censored (bit 1 lower, bit 2 upper), any of them may be NULL.  The CI is
 * computed by the device kernel behind plk_profile_ci_device: the call copies
 * the G values to the current device (allocating 8 (2G + 4) bytes there for
 * the call) and blocks until the result is back.  Errors: PLK_E_INVALID (G < 1,
 * NULL input, level outside (0, 1)), PLK_E_CUDA. */
plk_status plk_profile_ci(const double *grid, const double *profile_logL, int64_t G, double level, double *lo,
                          double *hi, double *argmax, int32_t *censored);

/* chi2_1 quantile used by the CI: c with P(chi2_1 <= c) = level. */
double plk_chi2_1_quantile(double level);

/* ------------------------------------------------------------------------ */
/* Post-processing of the Table-1 statistics (Sections 3.2, 3.4-3.6)          */
/* ------------------------------------------------------------------------ */

/* Statistics of K points of one dataset, as plk_eval_device writes them. */
typedef struct {
    int64_t n;               /* sites, n > p */
    int32_t p;               /* covariates, 1 <= p <= 16 */
    int32_t M;               /* lambda values, M >= 1, M + p <= 64 */
    int64_t K;               /* parameter points, >= 0 */
    const double *y;         /* device, n observations (> 0): the Box-Cox Jacobian's sum log y */
    const double *lambdas;   /* device, M */
    const double *ssq_yx;    /* device, K x (M+p) x (M+p) (plk_eval_args.ssq_yx) */
    const double *logdet;    /* device, K x 2 (only [k][0] = log|V| is read) */
    const int32_t *status;   /* device, K, or NULL: a point is used when (status & 15) == 0 */
} plk_stats_args;

/* Profile log-likelihood of one regression coefficient beta_j (Section 3.4,
 * eq. profilebetai), for each of the G grid values b = grid[g]:
 *   prof[g] = max over the used points k and all lambdas m of
 *             l(beta_j = b, beta_-j-hat(b), sigma-hat(b), omega_k, lambda_m),
 * where beta_-j-hat(b) and sigma-hat^2(b) = RSS(b)/n are the ML estimates of
 * the model with the offset X_j b (GLS of y' - X_j b on X_-j):
 *   -2 l = n log(RSS(b)/n) + log|V| - 2(lambda-1) sum log y + n log(2 pi) + n.
 * The ML form whatever the reml option of the evaluation was (the statistics
 * do not depend on it).  prof: device, G doubles, NaN where no pair gives a
 * finite value.  0 <= j < p.  grid, prof: device.  Runs on `stream`.
 * Errors: PLK_E_INVALID (sizes, NULL pointers, j), PLK_E_CUDA. */
plk_status plk_profile_beta_device(const plk_stats_args *stats, int32_t j, const double *grid,
                                   int64_t G, double *prof, void *stream);

/* The same profile with the REML criterion (Appendix, the subsection on beta_p
 * with REML, eq. remlprofileytilde):
 *   -2 l* = (n-p) log(RSS(b)/(n-p)) + log|V| + log|X^T V^-1 X|
 *           - 2(lambda-1) sum log y + n log(2 pi) + n - p,
 * RSS(b) as above and log|X^T V^-1 X| of the full X, as printed (stats->logdet
 * [k][1] is read as well).  Arguments and errors as plk_profile_beta_device. */
plk_status plk_profile_beta_reml_device(const plk_stats_args *stats, int32_t j, const double *grid,
                                        int64_t G, double *prof, void *stream);

/* Profile log-likelihood of sigma (Section 3.5, eq. profileSigma) at the G
 * grid values s = grid[g] (standard deviations, > 0; other values give NaN):
 *   prof[g] = max over the used points and all lambdas of
 *   -(1/2) [RSS/s^2 + n log s^2 + log|V| - 2(lambda-1) sum log y + n log(2 pi)],
 * RSS the residual sum of squares at beta-hat (Table 1 ssqResidual).  ML form.
 * Device pointers, `stream`; errors as plk_profile_beta_device. */
plk_status plk_profile_sigma_device(const plk_stats_args *stats, const double *grid, int64_t G,
                                    double *prof, void *stream);

/* Profile of lambda (Section 3.6): prof[m] = max over k of logL[k*M + m],
 * NaN values skipped (NaN if all are).  logL: device K x M (plk_eval_args.logL);
 * prof: device M.  1 <= M <= 65535.  The CI over the lambda grid then follows
 * from plk_profile_ci_device. */
plk_status plk_profile_lambda_device(const double *logL, int64_t K, int32_t M, double *prof,
                                     void *stream);

/* 1-D profile of any coordinate of the point cloud by its upper convex hull
 * (Section 3.6): the cloud is (x[k * x_stride], v[k]) for k < K (e.g. x = one
 * column of the K x 5 parameter rows with x_stride 5, v = the max over lambda
 * from plk_profile_max_device(logL, K, M, v)); points with a non-finite
 * coordinate are ignored.  Writes
 *   on_hull[k] = 1 if point k is a vertex of the upper hull, else 0 (device, K;
 *                required).  Per distinct x only the largest v can be a vertex
 *                (lowest k among equal values); points on a hull edge are not
 *                vertices;
 *   out[t]     = the linear interpolation of the vertices at xq[t] (device, Q),
 *                NaN outside the vertices' x range.
 * Work O(K^2) for the vertices, O(Q K) for the queries.  Runs on `stream`. */
plk_status plk_profile_hull_device(const double *x, int64_t x_stride, const double *v, int64_t K,
                                   const double *xq, int64_t Q, double *out, int32_t *on_hull,
                                   void *stream);

/* Internal parameters omega' = (gamma_1, kappa~, nu, gamma_2, gamma_3) of K
 * natural parameter rows (Section 3.2): gamma_1 = log phi_X + log phi_Y;
 * kappa~ = log kappa, or 1/sqrt(kappa) when kappa_hat_large != 0 (the MLE of
 * kappa is 4 or more); nu = sqrt(nu^2); gamma_2, gamma_3 = sqrt(phi_X/phi_Y - 1)
 * (cos 2 phi_A, sin 2 phi_A).  A ratio phi_X/phi_Y below one is first written
 * with the axes exchanged, (phi_Y, phi_X, phi_A + pi/2), the same correlation,
 * which negates (gamma_2, gamma_3).  params, out: device K x 5. */
plk_status plk_internal_params_device(const double *params, int64_t K, int32_t kappa_hat_large,
                                      double *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Instrumentation (not part of the paper's method)                          */
/* ------------------------------------------------------------------------ */

/* Per kernel class c < n_classes: total device milliseconds and launch count of
 * the launches made with PLK_FLAG_KERNEL_TIMING since the last reset.  Waits
 * for the recorded events (so call it after the work completes).  Returns the
 * number of classes the library defines in *n_defined when non-NULL.  reset != 0
 * clears the accumulators afterwards.  Process-wide, thread-safe. */
plk_status plk_kernel_timing(double *total_ms, int64_t *launches, int32_t n_classes, int32_t reset,
                             int32_t *n_defined);

/* Name of kernel class c ("" if out of range). */
const char *plk_kernel_class_name(int32_t c);

#ifdef __cplusplus
}
#endif
#endif /* PLK_H */

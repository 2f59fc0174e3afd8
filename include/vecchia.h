/*
 * vecchia.h -- C ABI of the GB300 (sm_103a) Vecchia likelihood library.
 *
 * The library evaluates, on one GPU, the Vecchia-approximate Gaussian-process
 * loglikelihood with the regression coefficients beta profiled out, its gradient and
 * its Fisher information with respect to the covariance parameters (James & Guinness,
 * "Implementation and Analysis of GPU Algorithms for Vecchia Approximation":
 * Sec. 2.1 Eq. 3 for the approximation, Algorithm 1 for the per-observation sums,
 * Sec. 3 for the profile step that turns the sums into loglik / gradient / information),
 * and runs Fisher scoring (Eq. 4) on top of it.
 *
 * Conventions shared by every entry point
 *   - Arrays are contiguous, row-major, 0-based.  Floating point arrays are FP64.
 *   - locs    n x d   observation locations (the order defines the Vecchia ordering).
 *   - y       n       responses.
 *   - X       n x p   design matrix (p >= 1; a column of ones for an intercept).
 *   - NNarray n x (m+1), int32.  Row i = [i, j_1, ..., j_k, -1, ..., -1]: column 0 is i
 *             itself, then the k = min(i, m) (or fewer) neighbours, all < i, then -1
 *             padding (Sec. 3: "row i containing the indices of the min(i, m+1)
 *             observations that are closest to observation i, including i itself").
 *             The neighbour order within a row does not change the result beyond rounding.
 *   - covparms, in this order (all > 0; the nugget variance is sigma2 * tau2, added on the
 *     diagonal only, as in Sec. 4.3 Eq. 5):
 *       VEC_EXP_ISO        (sigma2, rho, tau2)       C = sigma2 exp(-|h| / rho)         Eq. 6
 *       VEC_MATERN_ISO     (sigma2, rho, nu, tau2)   C = sigma2 2^(1-nu)/Gamma(nu) x^nu K_nu(x),
 *                                                    x = |h| / rho, 0.05 <= nu <= 20
 *       VEC_EXP_SPACETIME  (sigma2, rho_s, rho_t, tau2), d = 3 (lon, lat, time):
 *                          C = sigma2 exp(-sqrt((dlon^2 + dlat^2)/rho_s^2 + dt^2/rho_t^2))
 *       VEC_EXP_ANISO      (sigma2, rho_1, ..., rho_d, tau2), 1 <= d <= 20: one range per
 *                          coordinate, C = sigma2 exp(-sqrt(sum_k (h_k / rho_k)^2))
 *                          (Sec. 4.3, the form fitted to the Elevators attributes)
 *     The isotropic families take 1 <= d <= 3.
 *   - Results: loglik (scalar), grad (q), info (q x q, row-major, symmetric), betahat (p),
 *     where q = vecchia_nparms_d(covfun, d).  The loglikelihood includes -n/2 log(2 pi).
 *   - Errors are returned as vec_status codes; nothing is printed, no exception crosses
 *     the ABI, and the library never aborts the process.  vecchia_last_error() returns a
 *     thread-local message for the last failing call on the calling thread.
 */
#ifndef VECCHIA_GB300_H
#define VECCHIA_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define VECCHIA_API __attribute__((visibility("default")))
#else
#define VECCHIA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VEC_OK = 0,
    VEC_ERR_ARG = 1,         /* invalid argument or NNarray row                          */
    VEC_ERR_NOT_PD = 2,      /* a conditioning block is not positive definite            */
    VEC_ERR_NONFINITE = 3,   /* a non-finite value reached the sums                      */
    VEC_ERR_NOMEM = 4,       /* device allocation failed                                 */
    VEC_ERR_CUDA = 5,        /* a CUDA runtime call failed                               */
    VEC_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                            */
    VEC_ERR_UNSUPPORTED = 7  /* size or option outside what this library supports        */
} vec_status;

typedef enum {
    VEC_EXP_ISO = 0,
    VEC_MATERN_ISO = 1,
    VEC_EXP_SPACETIME = 2,
    VEC_EXP_ANISO = 3
} vec_covfun;

/* VEC_FP64: every step in FP64.  VEC_MIXED: covariance assembly, Cholesky trailing
 * updates and solves in FP32; pivots, per-observation last-row terms, the sums over
 * observations, the profile step and the Fisher step in FP64. */
typedef enum { VEC_FP64 = 0, VEC_MIXED = 1 } vec_precision;

/* Opaque context bound to one CUDA device.  It owns the library's device scratch
 * (per-block partial sums, the Matern coefficient table, fit state) and a CUDA stream
 * used by the synchronous entry points.  A handle may be used by one host thread at a
 * time; calls on one handle must not overlap on the GPU. */
typedef struct vec_handle_s* vec_handle;

/* Creates a handle on `device` (a CUDA ordinal).  Returns VEC_ERR_CUDA if the device
 * cannot be used.  *out is set to NULL on failure. */
VECCHIA_API vec_status vecchia_create(vec_handle* out, int device);

/* Frees the handle and its device scratch after synchronising its work. NULL is a no-op. */
VECCHIA_API vec_status vecchia_destroy(vec_handle h);

/* Message for the last error raised on the calling thread ("" if none). */
VECCHIA_API const char* vecchia_last_error(void);

/* Number of covariance parameters q of a covariance function whose count does not depend
 * on the dimension, or -1 (unknown, or VEC_EXP_ANISO: use vecchia_nparms_d). */
VECCHIA_API int vecchia_nparms(vec_covfun covfun);

/* Number of covariance parameters q of a covariance function on d-dimensional locations
 * (VEC_EXP_ANISO: d + 2), or -1 if the family is unknown or does not take d. */
VECCHIA_API int vecchia_nparms_d(vec_covfun covfun, int d);

/* Largest m this library supports (the conditioning block is (m+1) x (m+1)). */
VECCHIA_API int vecchia_max_m(void);

/* Lanes of a warp that work on one observation in the pass kernel: 1, 2, 4, 8, 16 or 32,
 * or 0 to let the library choose from the block size (the default).  A choice whose
 * shared-memory footprint does not fit makes later passes return VEC_ERR_UNSUPPORTED. */
VECCHIA_API vec_status vecchia_set_lanes(vec_handle h, int lanes);

/* Threads per block of the pass kernel: 32, 64, 96, 128, 192 or 256, or 0 to let the
 * library choose (the default).  Same rules as vecchia_set_lanes. */
VECCHIA_API vec_status vecchia_set_block_threads(vec_handle h, int threads);

/* Grouped conditioning only (vecchia_grouped_loglik_grad_info): how many members of a
 * group have their derivative terms formed together, 1..8, or 0 for the library's choice
 * (the default: the most, up to 4, whose slots fit).  More members per step give each
 * barrier more work but larger slots, hence fewer resident groups.  A choice whose slots
 * do not fit makes later grouped passes return VEC_ERR_UNSUPPORTED. */
VECCHIA_API vec_status vecchia_set_group_chunk(vec_handle h, int chunk);

/* Where the pass kernels read the per-pass Matern coefficient table: 1 = staged in shared
 * memory by every block, 0 = global memory (read through L1, which leaves more shared
 * memory for observation slots), -1 = the library's choice (the default: the autotuned
 * placement when a record matches, else shared memory when it fits).  Same rules as
 * vecchia_set_lanes; a placement that leaves no mapping fitting is ignored. */
VECCHIA_API vec_status vecchia_set_matern_table(vec_handle h, int placement);

/*
 * Autotuning of the kernel mapping.  vecchia_autotune runs the pass on the given inputs
 * (DEVICE pointers, as for vecchia_loglik_grad_info) once per candidate mapping -- lanes
 * per observation 1..32 x threads per block 64, 96, 128, 192, 256, every pair whose shared
 * memory fits -- times each with CUDA events (one warm-up, best of `reps`), and records the fastest in
 * the handle under the key (covfun, m, d, p, precision, floor(log2 n)).  Later passes and
 * fits on the handle whose key matches use that mapping unless vecchia_set_lanes /
 * vecchia_set_block_threads force one.  Outputs (HOST, may be NULL): the chosen lanes,
 * threads and its pass time in ms.  Synchronises `stream`.  Must not be called during a
 * stream capture.
 */
VECCHIA_API vec_status vecchia_autotune(vec_handle h, const double* locs, const double* y,
                                        const double* X, const int32_t* NNarray, int64_t n,
                                        int d, int p, int m, const double* covparms,
                                        vec_covfun covfun, vec_precision prec, void* stream,
                                        int reps, int* lanes_out, int* threads_out,
                                        float* ms_out);

/* Writes / reads the handle's autotuning records as JSON (an array of objects with keys
 * covfun, m, d, p, prec, log2n, lanes, threads, ms; prec is the vec_precision, plus 2 for
 * records of the batched pass).  Loading adds to the records. */
VECCHIA_API vec_status vecchia_autotune_save(vec_handle h, const char* path);
VECCHIA_API vec_status vecchia_autotune_load(vec_handle h, const char* path);

/* Tracing.  With timing enabled, every pass records CUDA events (on the pass's stream)
 * around its three phases: setup (status reset, Matern table), the per-observation kernel,
 * and the reduction + profile kernel.  vecchia_last_timing waits for the last traced pass
 * and returns the three durations in milliseconds (any pointer may be NULL); it returns
 * VEC_ERR_ARG if no traced pass has run.  Timing adds two event records per phase. */
VECCHIA_API vec_status vecchia_set_timing(vec_handle h, int enable);
VECCHIA_API vec_status vecchia_last_timing(vec_handle h, float* ms_setup, float* ms_pass,
                                           float* ms_profile);

/* Number of kernels one FP64 vecchia_loglik_grad_info call launches for this covariance
 * function (status reset, coefficient table, pass, sums of the block records, profile
 * step; used to count launches in benchmarks), or -1 for an unknown function. */
VECCHIA_API int vecchia_kernels_per_pass(vec_covfun covfun);

/*
 * vecchia_loglik_grad_info -- one Vecchia likelihood pass on device-resident data.
 *
 * Algorithm 1 (all n observations, including the first m, which condition on fewer
 * neighbours) followed by the profile step of Sec. 3:
 *   betahat = XSX^-1 ySX,
 *   loglik  = -n/2 log(2 pi) - 1/2 logdet - 1/2 (ySy - ySX' betahat),
 *   grad_j  = -1/2 (dlogdet_j + dySy_j - 2 betahat' dySX_j + betahat' dXSX_j betahat),
 *   info    = sum over observations of I(block) - I(neighbours).
 *
 * Pointers locs, y, X, NNarray, covparms: DEVICE memory on the handle's device, caller
 * owned, read only.  out: DEVICE memory, caller owned, length 1 + q + q*q + p doubles,
 * written as [loglik, grad[q], info[q*q], betahat[p]].  dev_status: DEVICE memory,
 * caller owned, 2 int64 values written as [vec_status, first failing observation or -1].
 * The call is asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream):
 * it returns after enqueuing.  The return value reports argument errors (VEC_ERR_ARG,
 * VEC_ERR_UNSUPPORTED) and launch failures (VEC_ERR_CUDA); errors found by the kernels
 * (bad NNarray row, covariance parameter out of range, block not positive definite,
 * non-finite sums) are reported in dev_status once the stream reaches that point, and
 * then out holds NaNs.  Requires 1 <= n < 2^31, 1 <= d <= 3 (d = 3 for the space-time
 * covariance, 1 <= d <= 20 for VEC_EXP_ANISO), 1 <= p <= 8, 0 <= m <= vecchia_max_m().
 */
VECCHIA_API vec_status vecchia_loglik_grad_info(vec_handle h, const double* locs, const double* y,
                                    const double* X, const int32_t* NNarray, int64_t n,
                                    int d, int p, int m, const double* covparms,
                                    vec_covfun covfun, vec_precision prec, void* stream,
                                    double* out, int64_t* dev_status);

/*
 * vecchia_loglik_grad_info_host -- the same pass end to end from HOST memory.
 *
 * All pointers are HOST memory, caller owned.  Inputs are copied to device buffers owned
 * by the handle (grown on demand, kept between calls), the pass runs on the handle's
 * stream, and the results are copied back before the call returns.  Outputs: *loglik,
 * grad[q], info[q*q], betahat[p]; *bad_index = first observation whose block is not
 * positive definite, or -1 (may be NULL).  Returns the kernel-side status as well
 * (VEC_ERR_NOT_PD, VEC_ERR_ARG for a bad NNarray row, ...).
 */
VECCHIA_API vec_status vecchia_loglik_grad_info_host(vec_handle h, const double* locs, const double* y,
                                         const double* X, const int32_t* NNarray, int64_t n,
                                         int d, int p, int m, const double* covparms,
                                         vec_covfun covfun, vec_precision prec,
                                         double* loglik, double* grad, double* info,
                                         double* betahat, int64_t* bad_index);

/*
 * vecchia_batch_loglik_grad_info -- the pass for many independent datasets at once.
 *
 * nbatch datasets share the covariance family, d and p; each has its own n_b, m_b and
 * theta_b.  Their arrays are concatenated: dataset b owns rows [off[b], off[b+1]) of locs,
 * y and X (off = point_offsets, HOST, nbatch+1 values, off[0] = 0), and its NNarray
 * (n_b x (m_b+1), indices LOCAL to the dataset, same conventions as above) follows the
 * previous dataset's in NNarray.  m: HOST, nbatch values.  covparms: DEVICE, nbatch x q.
 * out: DEVICE, nbatch x (1+q+q*q+p) doubles, row b = [loglik, grad, info, betahat] of
 * dataset b; dev_status: DEVICE, nbatch x 2 int64 ([status, first failing observation]).
 * One persistent launch covers all datasets: CTAs take tiles (ranges of observations of
 * one dataset) from a work counter, and each tile's sums form one record, so results do
 * not depend on the schedule.  The small work list (tiles, offsets) is copied from the
 * host first and the call waits for that copy; the pass itself is then enqueued on
 * `stream` and the call returns.  Requires 1 <= n_b, sum of n_b < 2^31,
 * 0 <= m_b <= vecchia_max_m().
 */
VECCHIA_API vec_status vecchia_batch_loglik_grad_info(
    vec_handle h, int nbatch, const double* locs, const double* y, const double* X,
    const int32_t* NNarray, const int64_t* point_offsets, const int* m, int d, int p,
    const double* covparms, vec_covfun covfun, vec_precision prec, void* stream, double* out,
    int64_t* dev_status);

/* Options of vecchia_fit.  A NULL pointer means the defaults shown. */
typedef struct {
    double tol;         /* stop when g~' I~^-1 g~ < tol on the log scale (1e-4)            */
    int maxit;          /* largest number of accepted Fisher steps (40, Table 2 of the paper)*/
    int max_halvings;   /* step halvings tried before giving up (10)                        */
    int use_graph;      /* 1: all iterations inside one CUDA graph with a WHILE node (1);
                           0: one host round trip per iteration                             */
    int prec;           /* VEC_FP64 (default): FP64 passes throughout.  VEC_MIXED: mixed-
                           precision passes until convergence, then FP64 passes from that
                           point until convergence again (the results are FP64 results).
                           VEC_FIT_MIXED_ONLY: mixed-precision passes throughout (the
                           optimum, loglik, gradient and information are the mixed path's) */
} vec_fit_opts;
#define VEC_FIT_MIXED_ONLY 2

/* Outcome of vecchia_fit. */
typedef struct {
    int status;         /* 0 converged, 1 iteration limit, 2 no ascent step, 3 start failed */
    int iters;          /* accepted Fisher steps (both phases for VEC_MIXED)                */
    int evals;          /* likelihood passes run (accepted steps + halvings + 1 per phase)  */
    int pass_status;    /* vec_status of the last pass                                      */
} vec_fit_info;

/*
 * vecchia_fit -- Fisher scoring (Eq. 4) for the covariance parameters, beta profiled.
 *
 * Iterates on log theta: g~ = theta (.) grad, I~ = diag(theta) info diag(theta),
 * Delta = I~^-1 g~ (a ridge r * 1e-4 * max diag(I~), r = 1..8, is added if I~ is not PD);
 * stops when g~' Delta < tol (checked before stepping) or after maxit accepted steps;
 * a trial theta (.) exp(Delta / 2^h) is accepted at the first h = 0..max_halvings whose
 * loglik is finite and larger; a failed pass counts as -inf; the Matern smoothness is
 * clamped to [0.05, 20].  Every iteration runs on the device (pass + step kernel); with
 * use_graph = 1 the whole loop is one CUDA graph launch.
 *
 * locs, y, X, NNarray: DEVICE memory (as in vecchia_loglik_grad_info).  start: HOST, q
 * values (must be valid parameters).  Outputs are HOST memory: theta_out (q), betahat (p),
 * *loglik, grad (q), info (q*q) at the final accepted parameters, and fit_info (may be
 * NULL).  Runs on `stream` and returns after the fit has finished.  Returns VEC_OK when
 * the loop ran (inspect fit_info->status), or an argument / CUDA error.
 */
VECCHIA_API vec_status vecchia_fit(vec_handle h, const double* locs, const double* y,
                                   const double* X, const int32_t* NNarray, int64_t n, int d,
                                   int p, int m, vec_covfun covfun, const double* start,
                                   const vec_fit_opts* opts, void* stream, double* theta_out,
                                   double* betahat, double* loglik, double* grad, double* info,
                                   vec_fit_info* fit_info);

/*
 * Batch plans: the batched pass split into a host-side preparation and a device-only run.
 *
 * vecchia_batch_plan_create does everything of vecchia_batch_loglik_grad_info that needs
 * the host: it checks the batch description (point_offsets and m, HOST, as there), splits
 * the datasets into up to three classes by block size (m + 1 <= 16, <= 32, larger; each
 * class is one launch whose shared-memory slots are sized for its own largest m), picks
 * each class's kernel mapping (forced on the handle, else the handle's batched autotuning
 * record for the class, else planned), builds the work list, allocates the plan's own
 * device buffers and uploads the work list (waiting for the copy).  The plan is bound to the handle's
 * device, independent of the handle afterwards, and must be released with
 * vecchia_batch_plan_destroy.
 *
 * vecchia_batch_plan_run enqueues one batched pass for the planned batch on `stream`:
 * the same arguments, layouts, results and per-dataset status as
 * vecchia_batch_loglik_grad_info, but it only launches kernels (no allocation, no copy,
 * no synchronisation), so it can be captured into a CUDA graph and replayed.  Runs of one
 * plan share its buffers: two runs of the same plan must not overlap on the GPU.
 *
 * vecchia_batch_plan_mapping reports the lanes per observation and threads per block of the
 * class with the most observations, and the number of tiles of all classes (HOST pointers,
 * each may be NULL).  vecchia_batch_plan_class reports class c (0, 1, 2: m + 1 <= 16,
 * <= 32, larger): its largest m (-1 for a class without datasets), lanes, threads and
 * tiles; VEC_ERR_ARG for c outside 0..2.
 */
typedef struct vec_batch_plan_s* vec_batch_plan;
VECCHIA_API vec_status vecchia_batch_plan_create(vec_handle h, int nbatch,
                                                 const int64_t* point_offsets, const int* m,
                                                 int d, int p, vec_covfun covfun,
                                                 vec_precision prec, vec_batch_plan* plan_out);
VECCHIA_API vec_status vecchia_batch_plan_run(vec_batch_plan plan, const double* locs,
                                              const double* y, const double* X,
                                              const int32_t* NNarray, const double* covparms,
                                              void* stream, double* out, int64_t* dev_status);
VECCHIA_API vec_status vecchia_batch_plan_mapping(vec_batch_plan plan, int* lanes, int* threads,
                                                  int* ntiles);
VECCHIA_API vec_status vecchia_batch_plan_class(vec_batch_plan plan, int c, int* mmax, int* lanes,
                                                int* threads, int* ntiles);
VECCHIA_API vec_status vecchia_batch_plan_destroy(vec_batch_plan plan);

/*
 * vecchia_batch_fit -- Fisher scoring (Eq. 4) for many independent datasets at once.
 *
 * Data as in vecchia_batch_loglik_grad_info (concatenated DEVICE arrays, HOST
 * point_offsets and m).  start: DEVICE, nbatch x q starting parameters (a dataset whose
 * start is not a valid parameter vector ends with status 3, start failed).  opts as in
 * vecchia_fit; every dataset follows the rules of vecchia_fit on its own, with its own
 * step, halvings and stopping test.  Each iteration is one batched pass (one persistent
 * launch) over the datasets that are still iterating, then one step kernel for all of
 * them; with use_graph = 1 the iterations run inside one CUDA graph whose WHILE node
 * repeats while any dataset iterates.  VEC_MIXED runs a mixed-precision phase for all
 * datasets, then an FP64 phase from each dataset's phase-1 result.
 * Outputs: theta_out, DEVICE, nbatch x q; out, DEVICE, nbatch x (1+q+q*q+p) = [loglik,
 * grad, info, betahat] at theta_out (FP64 pass values); fit_info, HOST, nbatch entries
 * (may be NULL).  Runs on `stream` and returns after all fits have finished.
 */
VECCHIA_API vec_status vecchia_batch_fit(vec_handle h, int nbatch, const double* locs,
                                         const double* y, const double* X,
                                         const int32_t* NNarray, const int64_t* point_offsets,
                                         const int* m, int d, int p, vec_covfun covfun,
                                         const double* start, const vec_fit_opts* opts,
                                         void* stream, double* theta_out, double* out,
                                         vec_fit_info* fit_info);

/*
 * vecchia_batch_autotune -- vecchia_autotune for the batched pass.
 *
 * For each class of datasets (by block size, as the batched pass splits them; see batch
 * plans) times the batched pass of that class's datasets (vecchia_batch_loglik_grad_info,
 * same arguments) under every (lanes per observation, threads per block) mapping that
 * fits the class's largest m, and records the fastest in the handle, keyed by (covfun,
 * the class's largest m, d, p, prec, floor(log2(the class's observations))) apart from the
 * single-dataset records; later batched calls whose classes match a key use it unless a
 * mapping is forced.  lanes_out and threads_out: the mapping of the class with the most
 * observations; ms_out: the sum of the classes' best times.  Synchronises `stream`.
 */
VECCHIA_API vec_status vecchia_batch_autotune(vec_handle h, int nbatch, const double* locs,
                                              const double* y, const double* X,
                                              const int32_t* NNarray,
                                              const int64_t* point_offsets, const int* m, int d,
                                              int p, const double* covparms, vec_covfun covfun,
                                              vec_precision prec, void* stream, int reps,
                                              int* lanes_out, int* threads_out, float* ms_out);

/*
 * Fields at shared locations.  nfields fields observed at the same n locations, with the
 * same covariates and NNarray (replicated simulations, the training fields of a learned
 * start): locs (n x d), X (n x p) and NNarray (n x (m+1)) are given once, Y is nfields x n
 * (row b = field b), covparms / start / theta_out are nfields x q.  All DEVICE memory.
 * Internally these are batches whose datasets share rows, so they run the same kernels
 * as the batched calls and return the same per-field results:
 *
 * vecchia_fields_loglik_grad_info -- as vecchia_batch_loglik_grad_info (out: nfields x
 *   (1+q+q*q+p), dev_status: nfields x 2).  Waits for the small work-list upload only.
 * vecchia_fields_fit -- as vecchia_batch_fit (fit_info: HOST, nfields entries or NULL).
 *   Returns after all fits have finished.
 * vecchia_fields_simulate -- draws from the Vecchia joint density the NNarray defines
 *   (Sec. 2.1, Eq. 3: each y_i given its listed earlier neighbours is Gaussian with the
 *   regression weights and conditional variance of the covariance model, nugget
 *   included): with b_i the last row of the inverse Cholesky factor of i's block
 *   (neighbours, then i), b_i . (y_N(i), y_i) = z_i, so y_i = (z_i - sum_c b_ic
 *   y_NN[i][c]) / b_i0 in the ordering.  z: nfields x n standard normal variates supplied
 *   by the caller; y: nfields x n output (mean zero: add X beta separately).  The factor
 *   rows are computed by the pass kernels in FP64 (a chunk of fields at a time, at most
 *   ~1 GiB of handle scratch), then one warp per field runs the recurrence.
 *   dev_status: nfields x 2 as for the pass (a block that is not positive definite, a bad
 *   NNarray row or bad parameters; y of such a field is undefined).  Asynchronous.
 */
VECCHIA_API vec_status vecchia_fields_loglik_grad_info(vec_handle h, int nfields,
                                                       const double* locs, const double* X,
                                                       const int32_t* NNarray, int64_t n, int d,
                                                       int p, int m, const double* Y,
                                                       const double* covparms, vec_covfun covfun,
                                                       vec_precision prec, void* stream,
                                                       double* out, int64_t* dev_status);
VECCHIA_API vec_status vecchia_fields_fit(vec_handle h, int nfields, const double* locs,
                                          const double* X, const int32_t* NNarray, int64_t n,
                                          int d, int p, int m, const double* Y, vec_covfun covfun,
                                          const double* start, const vec_fit_opts* opts,
                                          void* stream, double* theta_out, double* out,
                                          vec_fit_info* fit_info);
VECCHIA_API vec_status vecchia_fields_simulate(vec_handle h, int nfields, const double* locs,
                                               const int32_t* NNarray, int64_t n, int d, int m,
                                               const double* covparms, vec_covfun covfun,
                                               const double* z, void* stream, double* y,
                                               int64_t* dev_status);

/*
 * vecchia_fields_variogram -- binned empirical semivariogram features of fields at shared
 * locations (the input of a learned starting point for vecchia_fit; the paper has no
 * counterpart).
 *
 * For field f (row f of Y, nfields x n) the pairs are every (i, NNarray[i][c]), c >= 1,
 * NNarray[i][c] >= 0, and npairs random pairs (floor(r1 n / 2^32), floor(r2 n / 2^32))
 * from rand_pairs (DEVICE, 2 x npairs uint32, interleaved r1, r2; the same words for
 * every field).  A pair's squared lag h^2 = sum_k (s_ik - s_jk)^2 (FP64, coordinates in
 * order, no fused multiply-add) falls in bin k when edges2[k] <= h^2 < edges2[k+1]
 * (edges2: DEVICE, nbins + 1 ascending squared lags, 1 <= nbins <= 64); others are
 * ignored.  features (DEVICE, nfields x nbins, FP32): the mean of (y_i - y_j)^2 / 2 over
 * the bin's pairs, divided by the population variance of the field; an empty bin copies
 * the nearest non-empty bin (the lower one on a tie), all bins empty gives NaN.
 * bin_sum (FP64) and bin_count (int64), DEVICE nfields x nbins, may be NULL: the raw sums
 * and counts.  Sums are FP64 in a fixed order (deterministic).  Asynchronous on `stream`.
 */
VECCHIA_API vec_status vecchia_fields_variogram(vec_handle h, int nfields, const double* locs,
                                                const int32_t* NNarray, int64_t n, int d, int m,
                                                const double* Y, const uint32_t* rand_pairs,
                                                int64_t npairs, const double* edges2, int nbins,
                                                void* stream, float* features, double* bin_sum,
                                                int64_t* bin_count);

/*
 * Learned starting point for Fisher scoring (the paper has no counterpart; its fits start
 * from fixed rules).  A multilayer perceptron maps the 32 semivariogram features of a field
 * (vecchia_fields_variogram, 32 log-spaced lag bins) to the isotropic Matern parameters,
 * as the standardised targets (log(sigma2 / var y), log rho, log nu, log tau2):
 *   32 -> 128 (ReLU) -> 128 (ReLU) -> 4, FP32.
 * params: DEVICE, VEC_MLP_NPARAMS floats, row-major (out x in):
 *   W1[128][32], b1[128], W2[128][128], b2[128], W3[4][128], b3[4].
 * norm: DEVICE, VEC_MLP_NNORM floats: x_mean[32], x_std[32], t_mean[4], t_std[4]; the
 * network sees (x - x_mean) / x_std and its outputs are (t - t_mean) / t_std.
 *
 * vecchia_mlp_forward: out (nsamples x 4) = predictions o * t_std + t_mean for X
 *   (nsamples x 32).
 * vecchia_mlp_grad: loss = mean over samples and outputs of the squared error on the
 *   standardised targets T, and its gradient (VEC_MLP_NPARAMS floats).  The samples are
 *   rows index[0..nsamples) of X (rows x 32) and T (rows x 4), or rows 0..nsamples-1
 *   when index is NULL (a minibatch is a slice of a random permutation).
 * vecchia_mlp_adam_step: the same gradient, then one Adam step (beta1 0.9, beta2 0.999,
 *   eps 1e-8, bias corrections for step = 1, 2, ...) on params with the moment buffers
 *   adam_m, adam_v (VEC_MLP_NPARAMS floats each, zero before step 1); *loss (DEVICE, may be
 *   NULL) = the loss before the step.  Sums are in a fixed order: runs are reproducible.
 * vecchia_mlp_column_moments: column means and population standard deviations (1 where
 *   a column is constant) of X (rows x cols), for x_mean / x_std and t_mean / t_std.
 * vecchia_fields_warm_start: for fields at shared locations (as vecchia_fields_fit,
 *   MATERN_ISO), features (32 bins, squared edges edges2, random pairs as in
 *   vecchia_fields_variogram) -> network -> theta0 = (var(y) e^t0, e^t1, e^t2 clamped to
 *   [0.05, 20], e^t3); then one pass at theta0 and one at default_start (nfields x 4) in
 *   precision prec, and start (nfields x 4) = theta0 where it is finite, its pass
 *   succeeded and its loglik is not below the default's, else the default start.
 *   used_learned (nfields int) = 1 where theta0 was kept.  features (nfields x 32 FP32,
 *   may be NULL) receives the features.  Waits for the pass's work-list upload only.
 * All pointers DEVICE memory; asynchronous on `stream`.
 */
#define VEC_MLP_NPARAMS 21252
#define VEC_MLP_NNORM 72
VECCHIA_API vec_status vecchia_mlp_forward(vec_handle h, const float* params, const float* norm,
                                           const float* X, int nsamples, void* stream,
                                           float* out);
VECCHIA_API vec_status vecchia_mlp_grad(vec_handle h, const float* params, const float* norm,
                                        const float* X, const float* T, const int32_t* index,
                                        int nsamples, void* stream, float* grad, float* loss);
VECCHIA_API vec_status vecchia_mlp_adam_step(vec_handle h, float* params, float* adam_m,
                                             float* adam_v, int step, float lr,
                                             const float* norm, const float* X, const float* T,
                                             const int32_t* index, int nsamples, void* stream,
                                             float* loss);
VECCHIA_API vec_status vecchia_mlp_column_moments(vec_handle h, const float* X, int rows,
                                                  int cols, void* stream, float* mean,
                                                  float* sd);
/*
 * Small per-field steps of the learned start, on the device (all pointers DEVICE memory,
 * asynchronous on `stream`):
 * vecchia_fields_moments: mean and population variance (FP64, two passes, fixed-order
 *   sums) of each row of Y (nfields x n), the var(y) of the default start (Sec. 4's fit
 *   rules scale sigma2 by the data) and of the network's first output.
 * vecchia_mlp_targets: training targets (nfields x 4, FP32) from fitted parameters theta
 *   (nfields x 4, MATERN_ISO): (log(sigma2 / var), log rho, log nu, log tau2), component j
 *   clamped to [log lo[j], log hi[j]]; lo and hi are HOST arrays of 4 with
 *   0 < lo[j] <= hi[j] < inf.
 * vecchia_mlp_theta: theta0 (nfields x 4) from network outputs pred (nfields x 4, FP32):
 *   (var e^t0, e^t1, e^t2 clamped to [0.05, 20], e^t3), the rule vecchia_fields_warm_start
 *   applies.
 */
VECCHIA_API vec_status vecchia_fields_moments(vec_handle h, int nfields, int64_t n,
                                              const double* Y, void* stream, double* mean,
                                              double* var);
VECCHIA_API vec_status vecchia_mlp_targets(vec_handle h, int nfields, const double* theta,
                                           const double* var, const double* lo, const double* hi,
                                           void* stream, float* targets);
VECCHIA_API vec_status vecchia_mlp_theta(vec_handle h, int nfields, const float* pred,
                                         const double* var, void* stream, double* theta);
VECCHIA_API vec_status vecchia_fields_warm_start(vec_handle h, const float* params,
                                                 const float* norm, int nfields,
                                                 const double* locs, const double* X,
                                                 const int32_t* NNarray, int64_t n, int d, int p,
                                                 int m, const double* Y,
                                                 const uint32_t* rand_pairs, int64_t npairs,
                                                 const double* edges2,
                                                 const double* default_start,
                                                 vec_precision prec, void* stream, double* start,
                                                 int* used_learned, float* features);

/*
 * vecchia_ordered_nn -- the NNarray on the device.
 *
 * For an ordering of n locations (locs: DEVICE, n x d row-major FP64, already in the order
 * the likelihood will use, e.g. maxmin), row i of NNarray (DEVICE, n x (m+1) int32) is i
 * followed by its m nearest among locations 0..i-1, nearest first, -1 padded for i < m
 * (the input of vecchia_loglik_grad_info; the paper computes it on the CPU and names a GPU
 * version as future work).  Exact: the neighbours are the m smallest keys (d2, j) over
 * j < i in lexicographic order, d2 = the sum over coordinates, in order, of (x_ik -
 * x_jk)^2 with each product and sum rounded separately in FP64 (no fused multiply-add),
 * so ties go to the lower index and any FP64 implementation of the definition gives the
 * same array.  A uniform grid over the first two coordinates (built on the device) limits
 * the search; early observations, which have few earlier points, are searched by brute
 * force.  1 <= d <= 3, 0 <= m <= vecchia_max_m(), n < 2^31.  Handle scratch ~ 14 bytes
 * per location.  Asynchronous on `stream`.
 */
VECCHIA_API vec_status vecchia_ordered_nn(vec_handle h, const double* locs, int64_t n, int d,
                                          int m, void* stream, int32_t* NNarray);

/*
 * vecchia_maxmin_order -- the maxmin ordering on the device.
 *
 * order (DEVICE, n int64) receives the original indices of the n locations (locs: DEVICE,
 * n x d row-major FP64, 1 <= d <= 3) in maxmin order, the ordering Sec. 2.1 uses (the
 * paper computes it on the CPU): first the location nearest to the centroid, then at each
 * step the location whose smallest squared distance to the locations already chosen is
 * largest, ties to the lowest index.  Squared distances are sums over coordinates, in
 * order, of (x_k - y_k)^2 with every product and sum rounded separately in FP64, so the
 * decisions are those of any FP64 implementation of the definition; the centroid is a
 * fixed-order sum whose last bits may differ from another implementation's, which can
 * only matter when two locations are equally near it to within rounding.  Exact: each
 * step accepts the longest prefix of the candidates (sorted by distance, then index) that
 * the one-at-a-time rule would pick in a row.  One cooperative kernel runs all steps; its
 * grid barriers wait a bounded time and report VEC_ERR_TIMEOUT instead of hanging.
 * Handle scratch ~ 20 bytes per location.  Synchronises with `stream` before returning.
 */
VECCHIA_API vec_status vecchia_maxmin_order(vec_handle h, const double* locs, int64_t n, int d,
                                            void* stream, int64_t* order);

/*
 * vecchia_nearest -- the m nearest reference locations of each query location (for
 * prediction).  locs_ref: DEVICE nref x d, locs_query: DEVICE nquery x d (FP64, row-major);
 * NNarray: DEVICE nquery x m int32, row q = the indices of the m smallest keys (d2, j) over
 * all j < nref (d2 as in vecchia_ordered_nn), nearest first, -1 padded when nref < m.  Same
 * grid search as vecchia_ordered_nn.  1 <= m <= vecchia_max_m().  Asynchronous.
 *
 * vecchia_predict -- Vecchia prediction (kriging from a neighbour set).  For target q with
 * covariates X_pred[q] and neighbours NN_pred[q] (nquery x m rows of observation indices,
 * a valid prefix then -1, e.g. from vecchia_nearest):
 *   mean[q] = X_pred[q]' beta + k' Sigma_NN^-1 (y_N - X_N beta),
 *   var[q]  = c - k' Sigma_NN^-1 k,
 * Sigma_NN the covariance of the neighbours' observations (nugget sigma2 tau2 on its
 * diagonal), k their covariances with the target, and c = sigma2 when latent != 0 (the
 * latent field) or sigma2 (1 + tau2) (a new observation).  Computed per target from the
 * Cholesky factor of the (neighbours, target) block with one extra row of residuals, in
 * FP64.  All arrays DEVICE memory: locs (n x d), y (n), X (n x p), beta (p), locs_pred
 * (npred x d), X_pred (npred x p), NN_pred (npred x m), covparms (q); outputs mean, var
 * (npred) and dev_status (2: code, first failing target; VEC_ERR_NOT_PD if a block is not
 * positive definite, VEC_ERR_ARG for bad parameters or neighbour rows).  Asynchronous.
 */
VECCHIA_API vec_status vecchia_nearest(vec_handle h, const double* locs_ref, int64_t nref,
                                       const double* locs_query, int64_t nquery, int d, int m,
                                       void* stream, int32_t* NNarray);
VECCHIA_API vec_status vecchia_predict(vec_handle h, const double* locs, const double* y,
                                       const double* X, int64_t n, const double* beta,
                                       const double* locs_pred, const double* X_pred,
                                       const int32_t* NN_pred, int64_t npred, int d, int p,
                                       int m, const double* covparms, vec_covfun covfun,
                                       int latent, void* stream, double* mean, double* var,
                                       int64_t* dev_status);

/*
 * Grouped conditioning (Sec. 2.1, Sec. 5: one joint conditional per group).  Observations are
 * partitioned into groups that are contiguous ranges of the ordering; group b (members
 * B = s .. e-1) conditions jointly on U = (the members' NNarray neighbours) minus B, which
 * lies before s, so the product of the group conditionals p(y_B | y_U) is a valid density.
 * It equals the Vecchia density in which member i conditions on U and the earlier members
 * of its group, and it needs one Cholesky per group.
 *
 * vecchia_group_blocks -- HOST helper: the block lists from an NNarray (HOST, n x (m+1))
 * and group boundaries group_off (HOST, ngroups + 1, group_off[0] = 0, ascending,
 * group_off[ngroups] = n).  Block b is U (ascending) then the members s .. e-1:
 * block_idx[block_off[b] .. block_off[b+1]), nmemb[b] = e - s; *kmax = the largest block.
 * Call it first with block_idx = nmemb = NULL to get block_off and kmax (block_off[ngroups]
 * is the length block_idx needs), then with the arrays.  VEC_ERR_ARG on a bad NNarray row or
 * bad group boundaries.  No device work.
 *
 * vecchia_group_classes -- HOST helper: launch classes by block size.  Every slot of a
 * launch is sized for the launch's largest block, so blocks of very different sizes are
 * best run in separate launches.  From block_off (HOST, ngroups + 1) it picks at most nclass
 * (1..16) classes of block sizes minimising sum over classes of (groups x largest size^2)
 * (the slot size, hence the inverse occupancy) and writes gorder (HOST, ngroups: the group
 * indices, class by class; within a class by block size descending, then by index: the
 * grouped pass hands groups to its slots in this order, the quickest last), class_off
 * (HOST, nclass + 1: class c is gorder[class_off[c] .. class_off[c+1])) and class_kmax
 * (HOST, nclass: the class's largest block; unused trailing classes are empty with kmax 0).
 *
 * vecchia_grouped_loglik_grad_info -- the grouped pass: the same outputs as
 * vecchia_loglik_grad_info (loglik, gradient, Fisher information, betahat; n = the number
 * of observations, every one of them a member of exactly one group) from one group per
 * unit of work: the block's covariance and one Cholesky, then for each member row the
 * single-observation terms on the leading block that ends at that row.  DEVICE pointers:
 * locs, y, X as for the plain pass; block_off (ngroups + 1, int64), block_idx (int32),
 * nmemb (ngroups, int32) as vecchia_group_blocks writes them; gorder (ngroups, int32) as
 * vecchia_group_classes writes it, or NULL with nclass = 1 (groups in their own order).
 * HOST: class_off (nclass + 1), class_kmax (nclass), each class_kmax[c] in
 * [1, vecchia_max_m() + 1] for a non-empty class.  One kernel launch per non-empty class
 * (the largest blocks first), the launches side by side on `stream` and two side streams
 * of the handle that wait for `stream` and that `stream` then waits for (so the call is
 * ordered on `stream` like any other); each launch's slots take groups from a counter and
 * each group writes its own record, summed in group order (results do not depend on the
 * schedule); then one profile step.  Isotropic and space-time families
 * (VEC_ERR_UNSUPPORTED otherwise).  A block whose conditioning set is not ascending and
 * before its members, whose members are not consecutive, or longer than its class's
 * class_kmax, is reported in dev_status as VEC_ERR_ARG with the group index.  Asynchronous.
 */
VECCHIA_API vec_status vecchia_group_blocks(const int32_t* NNarray, int64_t n, int m,
                                            const int64_t* group_off, int64_t ngroups,
                                            int64_t* block_off, int32_t* block_idx,
                                            int32_t* nmemb, int* kmax);
VECCHIA_API vec_status vecchia_group_classes(const int64_t* block_off, int64_t ngroups,
                                             int nclass, int32_t* gorder, int64_t* class_off,
                                             int* class_kmax);
VECCHIA_API vec_status vecchia_grouped_loglik_grad_info(vec_handle h, const double* locs,
                                    const double* y, const double* X, int64_t n, int d, int p,
                                    int64_t ngroups, const int64_t* block_off,
                                    const int32_t* block_idx, const int32_t* nmemb,
                                    const int32_t* gorder, int nclass, const int64_t* class_off,
                                    const int* class_kmax, const double* covparms,
                                    vec_covfun covfun, vec_precision prec, void* stream,
                                    double* out, int64_t* dev_status);

/*
 * vecchia_measure_peaks -- throughputs of this GPU that bound the pass kernels, measured
 * on the handle's device and stream (synchronous, ~0.5 s): out[0] FP64 FMA-chain GFLOP/s,
 * out[1] FP32 FMA-chain GFLOP/s (8 independent chains per thread, 16 warps per SM),
 * out[2] exponential covariance evaluations per second (square root, exponential and
 * division per pair, as the pass does them), out[3] Matern evaluations per second (the
 * per-pass table's value and two derivatives), out[4] FP64 tensor-core GFLOP/s (chains of
 * the m8n8k4 double-precision matrix multiply-add, 8 per warp).  out: HOST memory,
 * 5 doubles.  Temporary device buffers are allocated and freed by the call.
 */
VECCHIA_API vec_status vecchia_measure_peaks(vec_handle h, double* out);

/*
 * vecchia_covariance_pairs -- the library's device covariance functions on explicit pairs.
 *
 * For each pair k: C[k] = C(la[k], lb[k]; covparms) including the nugget sigma2 tau2 when
 * same[k] != 0 (the two entries are the same observation), and dC[k*q + j] = dC/dtheta_j.
 * These are the functions assembled in Algorithm 1 (Sec. 4.3 Eq. 6 and the Matern family);
 * for the Matern family the call first rebuilds the handle's coefficient table for nu.
 * Pointers are DEVICE memory, caller owned: covparms (q), la and lb (npairs x d), same
 * (npairs int32), C (npairs), dC (npairs x q).  Asynchronous on `stream`.  covparms is
 * read on the device, so it is checked there: parameters outside the family's domain
 * (not positive and finite, or a Matern smoothness outside [0.05, 20]) give NaN in every
 * output entry.
 */
VECCHIA_API vec_status vecchia_covariance_pairs(vec_handle h, vec_covfun covfun, const double* covparms,
                                    int d, int64_t npairs, const double* la, const double* lb,
                                    const int32_t* same, double* C, double* dC, void* stream);

/*
 * vecchia_loglik_grad_info_noalloc -- the device-resident FP64 pass without any allocation.
 *
 * The paper has no counterpart to this entry point.  It is for callers that cannot
 * allocate device memory at the moment they need a likelihood value: programs whose GPU
 * memory is owned entirely by another allocator (a framework's caching pool, an
 * application that reserves the whole device at start-up) or held to a fixed budget, and
 * latency-sensitive loops that cannot afford the device-wide synchronisation an
 * allocation may cause.
 *
 * Arguments, layouts, results and error reporting are those of vecchia_loglik_grad_info
 * with prec = VEC_FP64, but there is no handle: it runs on the calling thread's current
 * CUDA device, all pointers must be device memory on that device, and the caller still
 * provides `out` and `dev_status`.  Only the FP64 path is offered: prec = VEC_MIXED is
 * rejected with VEC_ERR_UNSUPPORTED before anything runs.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch (per-block
 * partial sums, status word, Matern table) is one file-scope device array of
 * 1,102,592 bytes that every GPU loading this library holds until the process exits;
 * the partial-sum region holds 131072 doubles, and a pass whose launch plan needs more
 * (blocks x record length) is rejected with VEC_ERR_UNSUPPORTED before anything runs.
 * The first call on a device does a one-time set-up with that device current: it looks
 * up the array's device address (cudaGetSymbolAddress) and loads every kernel the entry
 * point can launch, so that later calls load no code.  Make that first call before any
 * stream capture.  Every call shares the one array and leaves its contents behind: the
 * kernels reset the status word and rewrite the rest in full on each call, but calls
 * whose work overlaps on the GPU (other streams, other host threads) race on it and must
 * be serialised.
 */
VECCHIA_API vec_status vecchia_loglik_grad_info_noalloc(const double* locs, const double* y,
                                                        const double* X, const int32_t* NNarray,
                                                        int64_t n, int d, int p, int m,
                                                        const double* covparms,
                                                        vec_covfun covfun, vec_precision prec,
                                                        void* stream, double* out,
                                                        int64_t* dev_status);

#ifdef __cplusplus
}
#endif

#endif /* VECCHIA_GB300_H */

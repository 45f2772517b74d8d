/*
 * sce.h -- C ABI of the GB300 (sm_103a) smoothed-circulant-embedding MLMC library.
 *
 * Method: Istratuca & Teckentrup, "Smoothed Circulant Embedding with
 * Applications to Multilevel Monte Carlo Methods for PDEs with Random
 * Coefficients".  Citations below name the paper's sections, equations and
 * algorithms.
 *
 * Conventions for every entry point
 *   - Return value: CE_OK (0) or a negative CE_ERR_* code.  No call throws,
 *     aborts or exits; ce_status_string() names a code.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it unless stated otherwise.
 *   - Array arguments marked "device" are caller-owned device memory
 *     (e.g. a torch tensor's data_ptr) on the current CUDA device; the library
 *     never frees them.  "host" arrays are caller-owned host memory.
 *   - Grids: an n-cell grid has (n+1) x (n+1) vertices x_p = p/n on [0,1]^2,
 *     stored row-major x-fastest: vertex (i, j) at index j*(n+1) + i (the
 *     lexicographic order of §2.1.2).  n must be a power of two, 4 <= n <= 4096.
 *   - Embedding side P = 2(n + J) is a power of two, 8 <= P <= 8192.
 *   - Handles are immutable after set-up: one handle may serve concurrent
 *     calls on several streams.
 */
#ifndef SCE_H
#define SCE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CE_OK = 0,
    CE_ERR_INVALID_ARG = -1,   /* bad size, NULL pointer, unsupported option   */
    CE_ERR_NOT_PSD = -2,       /* embedding not positive semi-definite          */
    CE_ERR_OOM = -3,           /* device or host allocation failed              */
    CE_ERR_CUDA = -4,          /* a CUDA runtime call failed                    */
    CE_ERR_NOT_CONVERGED = -5, /* at least one sample missed the tolerance      */
    CE_ERR_TIMEOUT = -6,       /* a bounded device wait gave up                 */
    CE_ERR_NONFINITE = -7      /* a non-finite value reached a result           */
};

enum { CE_COV_MATERN = 0, CE_COV_SEP_EXP = 1 };
enum { CE_PAD_NONE = 0, CE_PAD_DOUBLING = 1, CE_PAD_SMOOTH = 2 };

/* Covariance, §2.1: kind CE_COV_MATERN = Eq. (2.2) (nu in {0.5, 1.5, 2.5});
 * CE_COV_SEP_EXP = Eq. (2.3) with p = 1 (nu ignored). */
typedef struct {
    int kind;
    double nu, lambda, sigma2;
} ce_cov;

/* Padding, Algorithm 1 step 3(b) and §2.2.  mode CE_PAD_NONE: J as given,
 * CE_ERR_NOT_PSD if the check fails.  CE_PAD_DOUBLING: classical padding
 * (the covariance itself at the padded lags), P doubled until the check
 * passes.  CE_PAD_SMOOTH: smooth periodisation C_ext of Eq. (2.7) with
 * l = 1 + J/n, P doubled until the check passes.  J < 0 selects the default
 * (0 for NONE/DOUBLING, n for SMOOTH).  max_P bounds the search (<= 8192). */
typedef struct {
    int mode;
    int J;
    int max_P;
} ce_pad;

/* Smoothing, §2.4 and Algorithm 2 step 4(b): keep the `keep` largest
 * eigenvalues.  CE_KEEP_ALL (or any other negative value except
 * CE_KEEP_TAU_SQRT_S): all; CE_KEEP_TAU_SQRT_S: s - sqrt(s), i.e. drop
 * tau = sqrt(s) = P eigenvalues (the rule of the numerics of §4), resolved
 * once the padding has fixed P.  keep_fine shapes the fine field,
 * keep_coarse the coarse field of an MLMC level (read at every second
 * vertex).  A tie group (eigenvalues within tie_rel_tol relative of the cut
 * value) that straddles the cut is dropped whole.  tie_rel_tol <= 0 selects
 * 1e-10. */
enum { CE_KEEP_ALL = -1, CE_KEEP_TAU_SQRT_S = -2 };
typedef struct {
    long long keep_fine, keep_coarse;
    double tie_rel_tol;
} ce_smoothing;

typedef struct {
    int n, P, J;
    long long s;                              /* P*P                             */
    long long keep_eff_fine, keep_eff_coarse; /* eigenvalues kept after ties     */
    double lambda_min, lambda_max;            /* before clipping negatives to 0  */
    double max_imag;                          /* max |Im Lambda| (round-off)     */
} ce_embedding_info;

typedef struct ce_embedding_s *ce_embedding_t;

/*
 * ce_setup_embedding -- Algorithm 1 steps 1-3 (+ Algorithm 2 step 4(b)).
 * Builds the first column of the block-circulant embedding (§2.1.2, §2.2),
 * its eigenvalues Lambda = sqrt(s) F s by an FP64 2D FFT on the device
 * (Eq. (2.6) sign +i), checks min Lambda >= -1e-12 max Lambda (entries in
 * [-1e-12 max, 0) are clipped to 0), pads as `pad` says, and builds the
 * smoothing masks and the resident sqrt(Lambda~) tables (FP64 and FP32).
 *   cov, pad, sm : host structs (sm may be NULL = no smoothing)
 *   n            : cells per side of the field grid
 *   out          : host; receives a handle owning its device tables
 *   info         : host, may be NULL
 * Synchronises `stream` (reads back scalars).  Errors: CE_ERR_INVALID_ARG,
 * CE_ERR_NOT_PSD, CE_ERR_OOM, CE_ERR_CUDA.
 */
int ce_setup_embedding(const ce_cov *cov, int n, const ce_pad *pad, const ce_smoothing *sm,
                       void *stream, ce_embedding_t *out, ce_embedding_info *info);

/* Copies the P*P eigenvalues (after clipping, unmasked; index k1 + P*k2) to
 * dst (device if dst_on_device, else host; host copies synchronise). */
int ce_get_eigenvalues(ce_embedding_t e, double *dst, int dst_on_device, void *stream);

/* Copies the P*P fine (which = 0) or coarse (which = 1) keep-mask as bytes
 * (1 = kept) to host memory.  Synchronises. */
int ce_get_mask(ce_embedding_t e, int which, unsigned char *dst_host);

/*
 * ce_normals -- the normal generator of Algorithm 1 step 4(a) on its own:
 * out[c*len + j] = xi_j of sample first_sample + c, j < len (len a multiple
 * of 4).  Philox4x32-10 (Salmon et al., SC'11) with key (seed lo, seed hi),
 * counter (j/4, sample lo, sample hi, level); Box-Muller with the library's
 * IEEE-only ln/sin/cos.  precision 64: double out, u = (x + 0.5) 2^-32;
 * precision 32: float out, u = (float(x) + 0.5f) 2^-32.  out: device.
 */
int ce_normals(uint64_t seed, uint32_t level, uint64_t first_sample, int count, long long len,
               int precision, void *out, void *stream);

/*
 * ce_sample_batch -- Algorithm 1 step 4(a)-(f) (Algorithm 2 with masks) for
 * `count` samples first_sample .. first_sample+count-1 of MLMC level `level`:
 * xi (in registers) -> w = sqrt(Lambda~) xi -> v = F w (2D FFT, +i, unitary)
 * -> u = Re v + Im v -> Z = u on the (n+1)^2 grid -> k = exp(Z).
 *   precision 64: k arrays are double; 32: float (FP32 normals, FFT and exp).
 *   k_fine   : device, count*(n+1)^2, or NULL
 *   k_coarse : device, count*(n/2+1)^2, or NULL; the coarse field of the
 *              level (coarse mask), read at the even vertices of the grid
 * Errors: CE_ERR_INVALID_ARG, CE_ERR_OOM, CE_ERR_CUDA.
 */
int ce_sample_batch(ce_embedding_t e, uint64_t seed, uint32_t level, uint64_t first_sample,
                    int count, int precision, void *k_fine, void *k_coarse, void *stream);

/*
 * ce_sample_batch_noalloc -- the same fields as ce_sample_batch, for callers
 * that cannot allocate device memory per call: code that runs where
 * cudaMalloc/cudaMallocAsync is not allowed or not wanted, such as inside a
 * caller's own memory-pool or real-time budget, or a host framework that owns
 * all device allocation.  (The paper has no counterpart: this is a property of
 * the library, not of the method.)
 *   - Allocates nothing: the row/column intermediate lives in one fixed
 *     64 MiB device array inside the library (every device that loads the
 *     library reserves it until the process exits).  Batches are processed in
 *     chunks that fit the array; a single sample that does not fit
 *     ((n+1)*P complex values, plus (n/2+1)*P with a distinct coarse mask, in
 *     the chosen precision, must be <= 64 MiB) is rejected with
 *     CE_ERR_INVALID_ARG and a message in sce_last_error().
 *   - The first call on a device resolves the array's device address (a
 *     cudaGetSymbolAddress call, no allocation); make that first call before
 *     any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (other streams,
 *     other threads) race on it and must be serialised by the caller.
 *   - Uses the FFT launch shapes ce_autotune_fft chose, as ce_sample_batch
 *     does, so both entry points take the same time per chunk.
 *   - k_fine must not be NULL (k_coarse may be).  Other arguments, layouts and
 *     errors as ce_sample_batch.
 */
int ce_sample_batch_noalloc(ce_embedding_t e, uint64_t seed, uint32_t level,
                            uint64_t first_sample, int count, int precision, void *k_fine,
                            void *k_coarse, void *stream);

/*
 * ce_sample_levels -- the fields of several MLMC levels (Algorithm 1/2 step
 * 4(a)-(f), FP32) in one persistent kernel launch: the batching pattern for a
 * step that mixes levels of different grid sizes.  Each task is one
 * ce_sample_batch call (same handle, level, samples and outputs; a distinct
 * coarse mask gives the coarse field its own column pass), and its fields are
 * bit-identical to that call's.
 *   The launch's blocks take work items from a queue in device memory (one
 *   atomic counter): first every row-pass block of every task, then every
 *   column-pass block.  A column block of a sample waits until all row blocks
 *   of that sample are done (a per-sample counter); the wait is bounded by
 *   opts->wait_cycles SM clock cycles (default 2^31, about a second), after
 *   which the launch stops taking items and the call returns CE_ERR_TIMEOUT.
 *   A waiting block only depends on items handed out before its own, whose
 *   blocks never wait, so the launch needs no co-residency to finish.
 *   tasks : host array of ntasks (1..16) tasks; k_fine must not be NULL
 *   opts  : may be NULL.  opts->starve_task >= 0 makes that task's column
 *           blocks wait for one row block more than exist (a wait that runs
 *           out, for testing the timeout path); -1 = none.
 * Allocates the row/column intermediates of all tasks at once (stream
 * ordered) and synchronises `stream` to read the timeout flag.  Errors:
 * CE_ERR_INVALID_ARG, CE_ERR_OOM, CE_ERR_CUDA, CE_ERR_TIMEOUT.  Not a step of
 * the paper's method beyond the fields it computes.
 */
typedef struct {
    ce_embedding_t emb;
    uint32_t level;
    uint64_t first_sample;
    int count;
    void *k_fine;     /* device float, count*(n+1)^2 */
    void *k_coarse;   /* device float, count*(n/2+1)^2, or NULL */
} ce_field_task;

typedef struct {
    long long wait_cycles;   /* bound of a column block's wait; <= 0: default */
    int starve_task;         /* -1, or a task whose waits must run out (tests) */
} ce_levels_opts;

int ce_sample_levels(const ce_field_task *tasks, int ntasks, uint64_t seed,
                     const ce_levels_opts *opts, void *stream);

/* Darcy problem of §3.1, Eq. (3.1), on the n-cell grid:
 *   -div(k grad u) = f, u = 1 at x1 = 0, u = 0 at x1 = 1, zero flux at x2 = 0, 1;
 * P1 elements with nodal quadrature (§3.2; each cell split by the diagonal
 * (i,j)-(i+1,j+1), k averaged over each triangle's vertices).
 *   rtol      : relative residual target ||r|| <= rtol ||r_0|| (r_0 at u = lifting)
 *   maxit     : bound on preconditioned iterations (all inner iterations)
 *   precision : 64 = all-FP64 multigrid-preconditioned CG;
 *               32 = FP64 residual and solution with FP32 multigrid-CG
 *                    corrections (iterative refinement). */
typedef struct {
    int n;
    double f;
    double rtol;
    int maxit;
    int precision;
} darcy_problem;

/*
 * darcy_solve_batch -- solves the problem for `count` coefficient fields.
 *   k      : device, count*(n+1)^2, double if precision == 64 else float
 *   qoi    : device, count*3 doubles: [outflow through x1 = 1 (consistent
 *            flux), u(7/15, 7/15) (P1 interpolant), ||u_h||_L2 (P1 mass)]
 *   iters  : device int[count] or NULL: iterations used per sample
 *   status : device int[count] or NULL: 0 ok, CE_ERR_NOT_CONVERGED,
 *            CE_ERR_NONFINITE per sample
 *   u_out  : device double[count*(n+1)^2] or NULL: nodal solution
 * Returns CE_ERR_NOT_CONVERGED if any sample missed rtol (results are still
 * written).  Synchronises `stream` (reads back convergence counts).
 */
int darcy_solve_batch(const darcy_problem *p, const void *k, int count, double *qoi, int *iters,
                      int *status, double *u_out, void *stream);

/* Level sums of Algorithm 1/2 for one MLMC level (Eq. (3.5)). */
typedef struct {
    long long N;
    double sumY, sumY2, sumQf, sumQf2;
    int n_failed;
    int max_iters;          /* largest iteration count of one solve          */
    long long total_iters;  /* iterations summed over all fine + coarse solves */
} mlmc_level_sums;

/*
 * mlmc_level_estimate -- Algorithm 1 (Algorithm 2 with a smoothed handle):
 * for samples first_sample .. first_sample+count-1 of `level`, fields by
 * ce_sample_batch, Darcy solves on the fine grid and (level > 0) on the
 * coarse grid, QoI number qoi_index (0 outflow, 1 point value, 2 L2 norm),
 * Y = Q_f - Q_c (Y = Q_f on level 0), and the level sums (fixed-order
 * reduction on the device).  p->n must equal the handle's n; p->precision
 * selects the field and solver precision.
 *   out  : host, the level sums
 *   Y    : device double[count] or NULL
 *   qoi_f, qoi_c : device double[count*3] or NULL; when given, all three
 *          QoIs are computed for those solves, otherwise only qoi_index
 * Synchronises `stream`.  Returns CE_ERR_NOT_CONVERGED if any solve missed
 * rtol (sums still written; out->n_failed counts the samples).
 */
int mlmc_level_estimate(ce_embedding_t e, const darcy_problem *p, uint64_t seed, uint32_t level,
                        uint64_t first_sample, int count, int qoi_index, mlmc_level_sums *out,
                        double *Y, double *qoi_f, double *qoi_c, void *stream);

/*
 * One level's share of an MLMC step for mlmc_estimate_levels: the fields
 * of mlmc_level_estimate's arguments (emb, level, first_sample, count, Y,
 * qoi_f, qoi_c; same meaning and ownership) and its results.
 */
typedef struct mlmc_level_task {
    ce_embedding_t emb;
    uint32_t level;
    uint64_t first_sample;
    int count;
    double *Y;             /* device double[count] or NULL           */
    double *qoi_f, *qoi_c; /* device double[count*3] or NULL         */
    mlmc_level_sums sums;  /* out: the level sums                    */
    int status;            /* out: that level's mlmc_level_estimate status */
} mlmc_level_task;

/*
 * mlmc_estimate_levels -- all levels of one MLMC step (Eq. (3.5) needs the
 * level sums of every l = 0..L): each task computes exactly what
 * mlmc_level_estimate computes for it (bit-identical results), with p->n
 * taken from the task's handle.  With max_concurrency > 1 up to that many
 * levels run at once, each on its own CUDA streams driven by its own host
 * thread, the coarse solves of a level on a second stream; the largest
 * levels start first.  The streams start after the work queued on `stream`
 * and `stream` waits for all of them.  max_concurrency <= 1 runs the tasks
 * one after another on `stream`.  Synchronises the streams it uses.
 * Returns the first hard error of a task, else CE_ERR_NOT_CONVERGED if a
 * task reported it, else CE_OK; every task's own status is in its `status`.
 */
int mlmc_estimate_levels(const darcy_problem *p, uint64_t seed, int qoi_index,
                         mlmc_level_task *tasks, int ntasks, int max_concurrency, void *stream);

/*
 * mlmc_estimate_levels_persistent -- mlmc_estimate_levels with the fields of
 * every level generated first, in one persistent kernel launch on `stream`
 * (ce_sample_levels: a device work queue over all levels' row and column
 * blocks); then each level's solves, Y and sums as mlmc_estimate_levels runs
 * them.  Results are bit-identical to mlmc_estimate_levels.  FP32 path only
 * (p->precision == 32), 1..16 tasks, embeddings with P <= 4096.  Allocates
 * every level's fields at once (stream ordered).  Errors as
 * mlmc_estimate_levels, plus CE_ERR_TIMEOUT from the field launch.
 */
int mlmc_estimate_levels_persistent(const darcy_problem *p, uint64_t seed, int qoi_index,
                                    mlmc_level_task *tasks, int ntasks, int max_concurrency,
                                    void *stream);

/*
 * Request server -- MLMC level estimates (mlmc_level_estimate) served to
 * requests that arrive over time, with different grids and covariances, by
 * continuous batching.  `slots` host worker threads, each with its own
 * non-blocking CUDA stream on the device current at creation, admit queued
 * requests as soon as a slot is free and the request's device-memory
 * footprint (an upper bound of what its level estimate allocates) fits in
 * what is left of hbm_budget; admission is first-fit in arrival order, and
 * after 8 overtakes of a blocked head only the head is admitted.  Admitted
 * requests run concurrently.  Embedding set-ups are cached by (covariance,
 * n, padding, smoothing rule) and stay resident; unused ones are evicted
 * least-recently-used beyond max_embeddings.  A large request (above
 * slice_vertices) is cut into consecutive sample slices: at most two of its
 * slices are queued or running at a time, and each finished slice puts the
 * next one at the back of the queue, so requests that arrive meanwhile are
 * served between them.  The slices' level sums are added in slice order, so
 * a request's results do not depend on the other requests in the server:
 * they are bit-identical alone and in any mix (and, unsliced, bit-identical
 * to mlmc_level_estimate on its own).  Multigrid hierarchies are built per
 * sample from its own coefficient field inside each solve and cannot be
 * kept; what stays resident between requests are the embeddings.
 * The paper has no counterpart: this is how the level estimates of §3.4 are
 * served, not a step of the method.
 */
typedef struct sce_server_s *sce_server_t;

typedef struct {
    int slots;              /* requests in flight at once, 1..64                */
    long long hbm_budget;   /* bytes for admitted requests; <= 0: 3/4 of the
                               device memory free at creation                  */
    int max_embeddings;     /* resident embedding handles, >= 1                 */
    int precision;          /* 32 (FP32 field and MG, FP64 refinement) or 64    */
    double rtol;            /* FP64 residual tolerance of every solve           */
    int maxit;              /* CG iteration bound per solve                     */
    long long slice_vertices; /* a request of more than this many fine-grid
                               vertices of work (count * (n+1)^2) runs as
                               slices of samples that each stay within it; 0:
                               2^24; < 0: never sliced                         */
} sce_server_config;

typedef struct {
    ce_cov cov;
    ce_pad pad;
    int n;                  /* cells of the level's fine grid (power of two)    */
    uint32_t level;         /* MLMC level: > 0 adds the coarse solve on n/2     */
    int smoothing;          /* 0: full spectrum; 1: tau = sqrt(s) dropped (§4)  */
    int finest;             /* with smoothing: the fine field unsmoothed (§3.6) */
    uint64_t seed, first_sample;
    int count;              /* samples, >= 0                                    */
    int qoi_index;          /* 0 outflow, 1 point value, 2 L2 norm              */
    double f;               /* source term                                      */
    double *Y;              /* device double[count] or NULL; written when done  */
} sce_request;

typedef struct {
    mlmc_level_sums sums;   /* the level sums of the request's samples          */
    int status;             /* mlmc_level_estimate's status (or set-up error)   */
    int cache_hit;          /* 1: the embedding was resident                    */
    long long footprint;    /* bytes reserved at admission                      */
    double t_submit, t_admit, t_setup_done, t_done;  /* server clock, seconds   */
} sce_result;

typedef struct {
    long long submitted, completed, queued, in_flight, peak_in_flight;
    long long cache_hits, cache_misses, cached;
    long long reserved, peak_reserved, budget;   /* bytes                       */
    double now;                                  /* server clock, seconds       */
} sce_server_stats_t;

/* Starts the workers.  Errors: CE_ERR_INVALID_ARG, CE_ERR_OOM, CE_ERR_CUDA. */
int sce_server_create(const sce_server_config *cfg, sce_server_t *out);
/* Queues a request (copied; Y must stay valid until it is done) and returns
 * its ticket.  CE_ERR_INVALID_ARG for bad fields or a server shutting down. */
int sce_server_submit(sce_server_t s, const sce_request *r, uint64_t *ticket);
/* Waits up to timeout_s seconds (< 0: without limit) for the ticket; on
 * CE_OK fills *out and retires the ticket.  CE_ERR_TIMEOUT: not done yet
 * (the ticket stays valid).  CE_ERR_INVALID_ARG: unknown ticket. */
int sce_server_wait(sce_server_t s, uint64_t ticket, double timeout_s, sce_result *out);
int sce_server_stats(sce_server_t s, sce_server_stats_t *out);
/* Finishes every queued request, stops the workers, releases the cache. */
void sce_server_destroy(sce_server_t s);

/* Test hook (host side; not a step of the method): the next `count`
 * stream-ordered allocations of the library, in any thread, fail with
 * CE_ERR_OOM before reaching the CUDA allocator, to exercise the error paths
 * of the callers (the server's admission and recovery among them) without
 * exhausting device memory.  count <= 0 clears it. */
void sce_test_fail_allocs(int count);

/*
 * Quasi-Monte Carlo sampler (multilevel quasi-Monte Carlo, the outlook of
 * §5): the normals of Algorithm 1 step 4(a) replaced by a randomly shifted
 * rank-1 lattice rule with N points (a power of two, <= 2^31):
 *     y_j = frac((i z_r(j) mod N) / N + Delta_j),    xi_j = Phi^-1(y_j),
 * i = lattice point, r(j) = rank of frequency j = k1 + P k2 in increasing
 * wavenumber d(k1)^2 + d(k2)^2, d(k) = min(k, P-k), ties by j (low
 * frequencies carry the large eigenvalues of a decreasing spectral density;
 * an exact integer order, independent of eigenvalue rounding), z_r = a^r
 * mod N (Korobov vector, a odd), and Delta_j the uniform
 * shift (word + 0.5) 2^-32 of Philox4x32-10 with key (seed lo, seed hi) and
 * counter (j/4, shift, level, 0xFFFFFFFF), word j mod 4.  Each shift gives
 * an unbiased estimate; independent shifts estimate the error.  y is formed
 * exactly in FP64; Phi^-1 is evaluated on the smaller tail (symmetric).
 */
typedef struct ce_qmc_s *ce_qmc_t;

/* Builds the lattice table of handle e (P*P uint32 on the device; the handle
 * must outlive it).  Synchronises.  Errors: CE_ERR_INVALID_ARG (N not a power
 * of two or > 2^31, a even), CE_ERR_OOM, CE_ERR_CUDA. */
int ce_qmc_setup(ce_embedding_t e, uint32_t N, uint32_t a, ce_qmc_t *out);
void ce_qmc_destroy(ce_qmc_t q);

/* ce_sample_batch with the lattice normals of points first_point ..
 * first_point+count-1 (<= N) of shift `shift` on MLMC level `level`. */
int ce_sample_batch_qmc(ce_qmc_t q, uint64_t seed, uint32_t level, uint32_t shift,
                        uint32_t first_point, int count, int precision, void *k_fine,
                        void *k_coarse, void *stream);

/* mlmc_level_estimate with the lattice normals (same arguments and results;
 * the samples are lattice points first_point .. first_point+count-1 of one
 * shift). */
int mlmc_level_estimate_qmc(ce_qmc_t q, const darcy_problem *p, uint64_t seed, uint32_t level,
                            uint32_t shift, uint32_t first_point, int count, int qoi_index,
                            mlmc_level_sums *out, double *Y, double *qoi_f, double *qoi_c,
                            void *stream);

/*
 * Cached solvers and graphs.  With the environment variable SCE_GRAPHS=1 a
 * batched solve (darcy_solve_batch, and the solves of the MLMC calls) on a
 * stream other than the legacy default stream keeps its device buffers and a
 * CUDA graph of four captured CG iterations after it returns, in a pool of at
 * most 16 idle solvers per precision; a later solve with the same plan (sample
 * count, grid, window heights) on the same device takes them over and replays
 * the graph instead of launching the iterations one by one (the graph is
 * captured once per solver, on its first solve).  Results are identical to
 * the uncached path.  The pool holds device memory until this call frees it
 * (stream-ordered on `stream`, which it synchronises).  Not used while a
 * stream capture is in progress or the launch profiler is on.
 */
int darcy_solver_cache_clear(void *stream);

/*
 * darcy_autotune_tiles -- picks the window height (16, 24, 32, 48 or 64 rows; the
 * width is 64 columns) of the tiled multigrid kernels for grids of n cells
 * (n >= 128, a power of two) in `precision` by timing `reps` solves of
 * `count` samples of a smooth synthetic coefficient for every height (CUDA
 * events on `stream`, after one warm-up solve each).  The choice holds for
 * every later solve of the process in that precision whose hierarchy has an
 * n-cell level.  Tune the sizes in increasing order (a solve on n also runs
 * the levels below it).  Every height computes each vertex of a V-cycle
 * identically; the per-tile partial sums of r . z are added in an order that
 * follows the tiling, so solutions agree to rounding across heights (and
 * each height is deterministic).  Do not run other solves on
 * the device meanwhile (they would use the heights under trial).  The
 * environment variable SCE_TILE_SH, if set to one of the heights, overrides
 * every choice.  Not a step of the paper's method.
 *   height : host, may be NULL; receives the chosen height.
 * Errors: CE_ERR_INVALID_ARG (n not a power of two in [128, 4096], count not
 * in [1, 65535], reps < 1), CE_ERR_OOM, CE_ERR_CUDA.
 */
int darcy_autotune_tiles(int n, int precision, int count, int reps, void *stream, int *height);

/*
 * ce_autotune_fft -- picks the launch shapes (threads per FFT line, lines per
 * thread block) of the row and column passes of ce_sample_batch for handle
 * e's embedding size and `precision` by timing `reps` calls of `count`
 * samples for every admissible shape (CUDA events on `stream`), first for
 * the row pass, then for the column pass.  The choice holds for every later
 * call of the process with the same P and precision.  Every shape computes
 * each butterfly identically: tuning changes the time, never the fields.
 * Not a step of the paper's method.  Outputs (may be NULL): the chosen
 * shapes.  Synchronises `stream`.  Errors: CE_ERR_INVALID_ARG, CE_ERR_OOM,
 * CE_ERR_CUDA.
 */
int ce_autotune_fft(ce_embedding_t e, int precision, int count, int reps, void *stream,
                    int *row_tpf, int *row_F, int *col_tpf, int *col_F);

/*
 * Three-dimensional domains.  The paper writes the embedding (§2.1) and the
 * model problem (§3.1-3.2) for d <= 2 and states that higher dimensions
 * follow the same pattern; Eq. (2.7), the smoothing of §2.4 and its theorem
 * are stated for general d.  These entry points are the d = 3 instance:
 *   - grid: an n-cell grid has (n+1)^3 vertices p/n on [0,1]^3, vertex
 *     (i, j, k) at index (k*(n+1) + j)*(n+1) + i; n a power of two,
 *     2 <= n <= 256;
 *   - embedding side P = 2(n + J), a power of two, 4 <= P <= 512; s = P^3,
 *     array index k1 + P k2 + P^2 k3;
 *   - fields are FP32; the solver refines its FP32 multigrid-CG corrections
 *     against a float-float residual.
 */
typedef struct ce3_embedding_s *ce3_embedding_t;

/*
 * ce3_setup_embedding -- Algorithm 1 steps 1-3 in d = 3: first column
 * c[k3][k2][k1] = C_pad(d(k1)/n, d(k2)/n, d(k3)/n) (C_ext of Eq. (2.7) sums
 * the shifts in Z^3 with the cutoff of |x|_inf), Lambda = the unnormalised
 * +i DFT along the three axes in FP64, then the positivity check, padding
 * loop and smoothing masks of ce_setup_embedding.  CE_KEEP_TAU_SQRT_S drops
 * tau = floor(sqrt(s)) = floor(P^(3/2)) eigenvalues.  info->s = P^3.
 * Arguments, ownership and errors as ce_setup_embedding (max_P <= 512).
 */
int ce3_setup_embedding(const ce_cov *cov, int n, const ce_pad *pad, const ce_smoothing *sm,
                        void *stream, ce3_embedding_t *out, ce_embedding_info *info);
int ce3_get_info(ce3_embedding_t e, ce_embedding_info *info);
/* P^3 eigenvalues (clipped, unmasked), index k1 + P k2 + P^2 k3. */
int ce3_get_eigenvalues(ce3_embedding_t e, double *dst, int dst_on_device, void *stream);
/* P^3 keep-mask bytes, fine (which = 0) or coarse (1), to host memory. */
int ce3_get_mask(ce3_embedding_t e, int which, unsigned char *dst_host);
/* Releases the handle and its device tables (synchronises the device). */
void ce3_destroy(ce3_embedding_t e);

/*
 * ce3_sample_batch -- Algorithm 1 step 4 in d = 3 (Algorithm 2 with masks),
 * FP32, for samples first_sample .. first_sample+count-1 of `level`: xi_j,
 * j = k1 + P k2 + P^2 k3, is normal j of the sample's stream as ce_normals
 * with precision 32 -> w = sqrt(Lambda~) xi -> v = F w (threefold DFT, +i,
 * unitary) -> u = Re v + Im v on the (n+1)^3 grid -> k = exp(u).
 *   k_fine   : device float[count*(n+1)^3] or NULL
 *   k_coarse : device float[count*(n/2+1)^3] or NULL: the coarse field of
 *              the level (coarse mask) at the even vertices
 * Errors: CE_ERR_INVALID_ARG, CE_ERR_OOM, CE_ERR_CUDA.
 */
int ce3_sample_batch(ce3_embedding_t e, uint64_t seed, uint32_t level, uint64_t first_sample,
                     int count, float *k_fine, float *k_coarse, void *stream);

/*
 * darcy3_solve_batch -- -div(k grad u) = f on (0,1)^3, u = 1 at x1 = 0,
 * u = 0 at x1 = 1, zero flux on the other faces; P1 elements on the Kuhn
 * tetrahedra of each cell (the six simplices a, a+e_pi1, a+e_pi1+e_pi2,
 * a+(1,1,1), pi a permutation of the axes), k averaged over each
 * tetrahedron's four vertices (nodal quadrature).  Only axis-parallel edges
 * couple, so the operator is a seven-point stencil.  Solved by FP32
 * multigrid-preconditioned CG corrections of a float-float residual (FP32
 * pairs, ~48 significant bits; iterative refinement) to ||r|| <= rtol ||r_0||.
 *   p      : p->n as above, p->precision must be 32
 *   k      : device float[count*(n+1)^3]
 *   qoi    : device double[count*3]: [outflow through x1 = 1 (consistent
 *            flux), u(7/15, 7/15, 7/15) (P1 interpolant), ||u_h||_L2]
 *   iters, status, u_out : device or NULL, as darcy_solve_batch
 *            (u_out double[count*(n+1)^3])
 * Returns CE_ERR_NOT_CONVERGED if any sample missed rtol (results written).
 * Synchronises `stream`.
 */
int darcy3_solve_batch(const darcy_problem *p, const float *k, int count, double *qoi, int *iters,
                       int *status, double *u_out, void *stream);

/*
 * mlmc3_level_estimate -- Algorithm 1 (Algorithm 2 with a smoothed handle)
 * for one level in d = 3: fields by ce3_sample_batch, solves on the n- and
 * (level > 0) n/2-cell grids, Y = Q_f - Q_c of QoI qoi_index, level sums in
 * fixed order.  p->n must equal the handle's n.
 *   out : host, the level sums;  Y : device double[count] or NULL
 * Synchronises `stream`; CE_ERR_NOT_CONVERGED as mlmc_level_estimate.
 */
int mlmc3_level_estimate(ce3_embedding_t e, const darcy_problem *p, uint64_t seed, uint32_t level,
                         uint64_t first_sample, int count, int qoi_index, mlmc_level_sums *out,
                         double *Y, void *stream);

/* One level of an MLMC step in d = 3 for mlmc3_estimate_levels: the fields of
 * mlmc3_level_estimate's arguments (same meaning and ownership) and its results. */
typedef struct mlmc3_level_task {
    ce3_embedding_t emb;
    uint32_t level;
    uint64_t first_sample;
    int count;
    double *Y;             /* device double[count] or NULL           */
    mlmc_level_sums sums;  /* out: the level sums                    */
    int status;            /* out: that level's mlmc3_level_estimate status */
} mlmc3_level_task;

/*
 * mlmc3_estimate_levels -- all levels of one d = 3 MLMC step: each task
 * computes exactly what mlmc3_level_estimate computes for it (bit-identical),
 * with p->n taken from the task's handle.  With max_concurrency > 1 up to that
 * many levels run at once, each on its own CUDA stream driven by its own host
 * thread, largest levels first; the streams start after the work queued on
 * `stream` and `stream` waits for all of them.  max_concurrency <= 1 runs the
 * tasks one after another on `stream`.  Returns as mlmc_estimate_levels.
 */
int mlmc3_estimate_levels(const darcy_problem *p, uint64_t seed, int qoi_index,
                          mlmc3_level_task *tasks, int ntasks, int max_concurrency, void *stream);

/* Eq. (3.6): N_l = ceil(2 eps^-2 (sum_k sqrt(C_k V_k)) sqrt(V_l / C_l)),
 * l = 0..L.  V, C, N: host arrays of length L+1 (C > 0, V >= 0). */
int mlmc_optimal_samples(int L_plus_1, const double *V, const double *C, double eps, long long *N);

/*
 * The rules of §3.6 for the number of eigenvalues tau_l to drop on level l:
 * the tau at which the smoothing term of the level's error bound equals the
 * discretisation term C_alpha h_l^alpha.  The paper leaves the ratio
 * C_s / C_alpha to the user (cs_over_calpha > 0); alpha > 0 is the
 * discretisation rate.  Host-only (no device work); the result is real, the
 * caller rounds it to a count and passes s - tau as a keep count to
 * ce_setup_embedding (s is known once the padding loop has fixed P).
 *
 * mlmc_tau_exponential: separable exponential covariance (Eq. (2.3), p = 1)
 * without padding, s = 4 h^-2 (s >= 1): the closed form
 * tau = (s + 1) / ((C_s / (2^alpha C_alpha)) s^(alpha/2) + 1), not restricted
 * to [1, s].
 *
 * mlmc_tau_matern: Matern covariance (Eq. (2.2), nu > 0) under smooth
 * periodisation, s = 4 (1/h + J)^2 (h > 0, J >= 0): the root in [1, s] of
 * (s - tau + 1)^(-(1+nu)/2) tau = 2 (C_alpha / C_s) h^(alpha+1) (1/h + J),
 * clamped to 1 or s when the root lies outside.
 *
 * Both return CE_OK, or CE_ERR_INVALID_ARG for an argument outside the ranges
 * above or a NULL tau.
 */
int mlmc_tau_exponential(double s, double alpha, double cs_over_calpha, double *tau);
int mlmc_tau_matern(double h, double J, double nu, double alpha, double cs_over_calpha,
                    double *tau);

/* Releases a handle and its device tables (synchronises the device). */
void ce_destroy(ce_embedding_t e);

const char *ce_status_string(int status);

/* Text of the last CUDA runtime failure seen by the calling thread. */
const char *sce_last_error(void);

/*
 * Launch profiler -- instrumentation of this library, not a step of the
 * paper's method.  sce_profile_enable(1) clears the totals and records a CUDA
 * event pair around every subsequent kernel launch (on the launching stream),
 * per kernel family, together with the algorithmic bytes the library
 * attributes to that launch; sce_profile_enable(0) stops recording.
 * sce_profile_read waits for the recorded events and returns the family's
 * total elapsed milliseconds, algorithmic bytes and launch count (any
 * pointer may be NULL).  Families are numbered 0 .. sce_profile_count()-1
 * and named by sce_profile_name.  Not thread-safe against concurrent
 * enable/read calls.
 */
void sce_profile_enable(int on);
int sce_profile_read(int kernel, double *ms, double *bytes, long long *launches);
int sce_profile_count(void);
const char *sce_profile_name(int kernel);

/*
 * Machine peaks -- instrumentation of this library, not a step of the paper's
 * method: the denominators of the roofline fractions of kernels that HBM
 * bandwidth does not bound.  Both only launch one kernel on `stream`; the
 * caller times it with CUDA events on that stream.
 * sce_peak_fma: `blocks` blocks of 256 threads; every thread runs
 *   iters * 128 FP32 FMAs in eight independent chains, i.e.
 *   blocks * 8 * iters * 128 FMA warp instructions and
 *   blocks * 256 * iters * 256 FLOP in all.  out: device float[blocks],
 *   written only in a case that cannot occur (keeps the work live).
 * sce_peak_l2: `blocks` blocks of 256 threads read the device buffer `buf`
 *   (16-byte aligned, `bytes` a multiple of 16) `reps` times through L2 only
 *   (ld.global.cg), bytes * reps bytes in all; size it well below the L2
 *   capacity and discard the first launch so that the reads hit L2.
 *   out: device float[blocks], as above.
 * Errors: CE_ERR_INVALID_ARG for null pointers, non-positive counts or a
 * misaligned buffer; CE_ERR_CUDA if the launch fails.
 */
int sce_peak_fma(float *out, int blocks, int iters, void *stream);
int sce_peak_l2(const void *buf, size_t bytes, int reps, int blocks, float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SCE_H */

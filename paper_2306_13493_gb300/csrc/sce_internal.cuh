// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <vector>

#include "../../include/sce.h"

#define SCE_CUDA(call)                                                                  \
    do {                                                                                \
        cudaError_t err__ = (call);                                                     \
        if (err__ != cudaSuccess) {                                                     \
            sce_set_last_cuda_error(err__, #call, __FILE__, __LINE__);                  \
            return err__ == cudaErrorMemoryAllocation ? CE_ERR_OOM : CE_ERR_CUDA;       \
        }                                                                               \
    } while (0)

#define SCE_TRY(call)                   \
    do {                                        \
        int st__ = (call);                      \
        if (st__ != CE_OK) return st__;         \
    } while (0)

void sce_set_last_cuda_error(cudaError_t err, const char *what, const char *file, int line);

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static inline bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
static inline int ilog2(long long v) {
    int r = 0;
    while ((1LL << r) < v) ++r;
    return r;
}

// Raises the dynamic shared-memory limit of kernel `func` on the current
// device to at least `bytes`, never lowering it.  The limit is a process-wide
// attribute of the kernel: calls on several host threads with different sizes
// must not lower it between another thread's setting and its launch.
int sce_raise_smem_limit(const void *func, size_t bytes);

// Keep-mask of the smoothing step (Algorithm 2 step 4(b)) over the flattened
// eigenvalues L: the keep largest, a tie group straddling the cut dropped whole
// (relative tolerance tol).  keep < 0 or >= L.size(): all.  Returns the count kept.
long long sce_keep_mask(const std::vector<double> &L, long long keep, double tol,
                        std::vector<unsigned char> &mask);

// Stream-ordered device allocation from the device's default pool.
int sce_alloc(void **p, size_t bytes, cudaStream_t st);
int sce_free(void *p, cudaStream_t st);

template <typename T>
static inline int sce_alloc_t(T **p, size_t count, cudaStream_t st) {
    return sce_alloc(reinterpret_cast<void **>(p), count * sizeof(T), st);
}

// Twiddle tables exp(+2 pi i k / P), k = 0..P-1, built once per P and device.
const double2 *sce_twiddles64(int P, int *status);
const float2 *sce_twiddles32(int P, int *status);
// Lookup of already built tables (never allocates); CE_ERR_INVALID_ARG if absent.
int sce_twiddles_lookup(int P, const double2 **d64, const float2 **d32);
// Sets the text returned by sce_last_error().
void sce_set_last_error_text(const char *text);

struct ce_embedding_s {
    int device;
    int n, P, J, mode;
    ce_cov cov;
    long long s;
    long long keep_eff_fine, keep_eff_coarse;
    bool coarse_distinct;   // coarse mask differs from the fine mask
    double lambda_min, lambda_max, max_imag;
    double *lam;            // P*P eigenvalues (clipped), device
    double *sq64_f;         // P*P sqrt(Lambda~_fine), device
    double *sq64_c;         // P*P sqrt(Lambda~_coarse) (== sq64_f if !coarse_distinct)
    float *sq32_f;
    float *sq32_c;
    std::vector<unsigned char> mask_f, mask_c;   // host copies
};

// ---------------------------------------------------------------- profiling
// Kernel families timed by the optional launch profiler (sce_profile_*).
enum SceKernel {
    KP_ROW = 0, KP_COL, KP_COND, KP_COARSEN, KP_SMOOTH, KP_RESTRICT, KP_PROLONG, KP_COARSEST,
    KP_SPMV, KP_AXPY, KP_DOT, KP_PUPDATE, KP_COPY, KP_REDUCE, KP_OUTER_RES, KP_OUTER_UPD, KP_QOI,
    KP_SETUP, KP_NORMALS, KP_LEVEL, KP_SMALL, KP_MG_DOWN, KP_MG_UP, KP_MG_TAIL,
    // three-dimensional path
    KP_X3, KP_Y3, KP_Z3, KP_COND3, KP_SMOOTH3, KP_RESID3, KP_RESTRICT3, KP_PROLONG3, KP_SPMV3,
    KP_VEC3, KP_OUTER3, KP_MG_V64, KP_LEVELS, KP_COARSEN_TAIL, KP_MG_DOWN3, KP_MG_UP3,
    KP_COUNT_
};

bool sce_prof_on();
// Records a start event (when profiling is on) and, on destruction, the end
// event of the launch(es) enqueued in between; `bytes` = algorithmic bytes.
struct SceProf {
    int id = -1;
    int slot = -1;
    cudaStream_t st = nullptr;
    SceProf(int kernel, cudaStream_t s, double bytes);
    ~SceProf();
};

// A position in the launch records, and the correction of the bytes that the
// launches after it on stream st, of the families ids[0..nids), attributed to
// themselves: multiplied by f.  A kernel whose launch covers every sample but
// skips the converged ones (per-sample flags on the device) is charged the
// bytes of all samples when it is launched; the solver, which knows at its end
// how many sample-passes actually ran, scales them to those.  No effect while
// the profiler is off, or once the records were read since the mark.
struct SceProfMark {
    long long gen = -1, idx = 0;
};
SceProfMark sce_prof_mark();
void sce_prof_scale(const SceProfMark &m, cudaStream_t st, const int *ids, int nids, double f);

// Field path entry used by mlmc_level_estimate (same as ce_sample_batch).
// Lattice normals of the quasi-Monte Carlo sampler (ce_qmc_setup): for point i
// and grid index j, y = frac((i zr[j] mod N)/N + Delta_j), xi = Phi^-1(y), with
// Delta_j from Philox (counter (j/4, shift_sample, SCE_QMC_SHIFT_LEVEL)).
constexpr uint32_t SCE_QMC_SHIFT_LEVEL = 0xFFFFFFFFu;
struct QmcArgs {
    const uint32_t *zr;      // device, P*P: a^rank(j) mod N
    uint32_t N;              // points, a power of two
    uint64_t shift_sample;   // (level << 32) | shift
};
struct ce_qmc_s {
    ce_embedding_t e;
    uint32_t N, a;
    uint32_t *zr;
    int device;
};

// qa == nullptr: Philox normals (the Monte Carlo sampler); otherwise lattice
// point first_sample + c of the shift in qa.
int sce_sample_batch_impl(ce_embedding_t e, uint64_t seed, uint32_t level, uint64_t first_sample,
                          int count, int precision, void *k_fine, void *k_coarse, cudaStream_t st,
                          const QmcArgs *qa = nullptr);

// Relative residual drop each inner FP32 PCG solve of the mixed path aims
// for before the float-float refinement recomputes the residual
// (SCE_INNER_REL, default 2e-5).
double sce_inner_rel_f32();

// Padded rows (pitch n + 2) for the shared-memory levels of at least 32 cells:
// in the fused n = 64 cycle by default (SCE_SMEM_PAD=0: n + 1), in the
// one-block solvers with SCE_SMALL_PAD=1 (their CG loops then compute a row
// index per vertex, which measured slower than the bank conflicts it removes).
bool sce_smem_pad();
bool sce_small_pad();

// One-block-per-sample solver for small grids (mixed precision).  qmask bit 3:
// u_out holds float-float pairs (float2) instead of doubles.  u_init: NULL, or
// the solutions of the samples on the n/2 grid ((n/2+1)^2 per sample; float2
// pairs when u_init_ff, else doubles), prolonged bilinearly into the first
// iterate; the stopping rule stays relative to the lifting's residual.
int sce_small_max_n();
int sce_darcy_small(const darcy_problem *p, const float *k, int count, double *qoi, int *iters,
                    int *status, double *u_out, cudaStream_t st, int *max_iters_out,
                    int *n_failed_out, int qmask, const void *u_init = nullptr,
                    bool u_init_ff = false);

// Darcy solver entry used by mlmc_level_estimate.  max_iters_out, if not
// NULL, points at int[2]: {max iterations over the samples, total iterations}.
// qmask selects the QoIs computed (bit 0 outflow, 1 point value, 2 L2 norm;
// the others are written as 0).  u_init (device, count*(n/2+1)^2 doubles, or
// NULL = the lifting): the solution of the same field on the n/2-cell grid,
// whose bilinear prolongation is the batched solver's first iterate; the
// convergence test stays relative to the lifting's residual.  The one-block
// solver (small n) ignores it.  u_ff (FP32 problems only): u_out and u_init
// hold float-float pairs (float2, hi + lo) instead of doubles -- the mixed
// path's own representation, so the hand-over between the coarse and the fine
// solve of a level needs no FP64 arithmetic.
int sce_darcy_solve_impl(const darcy_problem *p, const void *k, int count, double *qoi, int *iters,
                         int *status, double *u_out, cudaStream_t st, int *max_iters_out,
                         int *n_failed_out, int qmask, const double *u_init = nullptr,
                         bool u_ff = false);

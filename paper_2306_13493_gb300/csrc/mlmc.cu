// One MLMC level of Algorithm 1 (Algorithm 2 with a smoothed handle):
// fields -> fine and coarse Darcy solves -> Y_l = Q_f - Q_c (Y_0 = Q_f) ->
// level sums (N, sum Y, sum Y^2, sum Q_f, sum Q_f^2) for Eq. (3.5).
#include <algorithm>
#include <vector>

#include "sce_internal.cuh"

namespace {

__global__ void level_diff_kernel(const double *__restrict__ qf, const double *__restrict__ qc,
                                  int count, int qi, double *__restrict__ Y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    Y[s] = qf[3 * s + qi] - (qc ? qc[3 * s + qi] : 0.0);
}

// One block, fixed-order: per-thread strided sums, then a shared-memory tree.
__global__ void level_sums_kernel(const double *__restrict__ Y, const double *__restrict__ qf,
                                  int count, int qi, double *__restrict__ out4) {
    __shared__ double sh[4][256];
    double a = 0, b = 0, c = 0, d = 0;
    for (int s = threadIdx.x; s < count; s += blockDim.x) {
        const double y = Y[s], q = qf[3 * s + qi];
        a += y;
        b += y * y;
        c += q;
        d += q * q;
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    sh[3][threadIdx.x] = d;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int r = 0; r < 4; ++r) sh[r][threadIdx.x] += sh[r][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out4[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

extern "C" int mlmc_level_estimate(ce_embedding_t e, const darcy_problem *p, uint64_t seed,
                                   uint32_t level, uint64_t first_sample, int count,
                                   int qoi_index, mlmc_level_sums *out, double *Y, double *qoi_f,
                                   double *qoi_c, void *stream) {
    if (!e || !p || !out || count < 0 || qoi_index < 0 || qoi_index > 2) return CE_ERR_INVALID_ARG;
    if (p->n != e->n || (p->precision != 32 && p->precision != 64)) return CE_ERR_INVALID_ARG;
    *out = mlmc_level_sums{};
    if (count == 0) return CE_OK;
    cudaStream_t st = as_stream(stream);
    const int n = e->n, nc = n / 2;
    const bool coarse = level > 0;
    const size_t es = p->precision == 64 ? sizeof(double) : sizeof(float);
    const long long Vf = (long long)(n + 1) * (n + 1), Vc = (long long)(nc + 1) * (nc + 1);
    // chunk: bound the number of fine vertices resident at once
    const long long max_vertices = 1LL << 27;
    int chunk = (int)std::max<long long>(1, std::min<long long>(count, max_vertices / Vf));
    chunk = std::min(chunk, 65535);

    void *kf = nullptr, *kc = nullptr;
    double *qf = nullptr, *qc = nullptr, *Yd = nullptr, *sums = nullptr;
    std::vector<void *> owned;
    auto cleanup = [&]() {
        for (void *q : owned) sce_free(q, st);
    };
    int rc = CE_OK;
    auto A = [&](void **ptr, size_t bytes) {
        int r = sce_alloc(ptr, bytes, st);
        if (r == CE_OK) owned.push_back(*ptr);
        return r;
    };
    if ((rc = A(&kf, (size_t)chunk * Vf * es)) != CE_OK) { cleanup(); return rc; }
    if (coarse && (rc = A(&kc, (size_t)chunk * Vc * es)) != CE_OK) { cleanup(); return rc; }
    if (!qoi_f && (rc = A((void **)&qf, (size_t)chunk * 3 * sizeof(double))) != CE_OK) { cleanup(); return rc; }
    if (coarse && !qoi_c && (rc = A((void **)&qc, (size_t)chunk * 3 * sizeof(double))) != CE_OK) { cleanup(); return rc; }
    if (!Y && (rc = A((void **)&Yd, (size_t)chunk * sizeof(double))) != CE_OK) { cleanup(); return rc; }
    if ((rc = A((void **)&sums, 4 * sizeof(double))) != CE_OK) { cleanup(); return rc; }

    darcy_problem pc = *p;
    pc.n = nc;
    double acc[4] = {0, 0, 0, 0};
    int n_failed = 0, max_it = 0;
    long long tot_it = 0;
    int result = CE_OK;
    for (int c0 = 0; c0 < count; c0 += chunk) {
        const int cn = std::min(chunk, count - c0);
        double *qf_c = qoi_f ? qoi_f + 3 * (size_t)c0 : qf;
        double *qc_c = coarse ? (qoi_c ? qoi_c + 3 * (size_t)c0 : qc) : nullptr;
        double *Y_c = Y ? Y + c0 : Yd;
        rc = sce_sample_batch_impl(e, seed, level, first_sample + (uint64_t)c0, cn, p->precision, kf,
                                   coarse ? kc : nullptr, st);
        if (rc != CE_OK) { cleanup(); return rc; }
        int mi[2] = {0, 0}, nf = 0;
        rc = sce_darcy_solve_impl(p, kf, cn, qf_c, nullptr, nullptr, nullptr, st, mi, &nf,
                                  qoi_f ? 7 : (1 << qoi_index));
        if (rc != CE_OK && rc != CE_ERR_NOT_CONVERGED) { cleanup(); return rc; }
        if (rc == CE_ERR_NOT_CONVERGED) result = rc;
        n_failed += nf;
        max_it = std::max(max_it, mi[0]);
        tot_it += mi[1];
        if (coarse) {
            rc = sce_darcy_solve_impl(&pc, kc, cn, qc_c, nullptr, nullptr, nullptr, st, mi, &nf,
                                      qoi_c ? 7 : (1 << qoi_index));
            if (rc != CE_OK && rc != CE_ERR_NOT_CONVERGED) { cleanup(); return rc; }
            if (rc == CE_ERR_NOT_CONVERGED) result = rc;
            n_failed += nf;
            max_it = std::max(max_it, mi[0]);
            tot_it += mi[1];
        }
        level_diff_kernel<<<(cn + 255) / 256, 256, 0, st>>>(qf_c, qc_c, cn, qoi_index, Y_c);
        level_sums_kernel<<<1, 256, 0, st>>>(Y_c, qf_c, cn, qoi_index, sums);
        if (cudaGetLastError() != cudaSuccess) { cleanup(); return CE_ERR_CUDA; }
        double h[4];
        if (cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cleanup();
            return CE_ERR_CUDA;
        }
        for (int r = 0; r < 4; ++r) acc[r] += h[r];
    }
    cleanup();
    out->N = count;
    out->sumY = acc[0];
    out->sumY2 = acc[1];
    out->sumQf = acc[2];
    out->sumQf2 = acc[3];
    out->n_failed = n_failed;
    out->max_iters = max_it;
    out->total_iters = tot_it;
    return result;
}

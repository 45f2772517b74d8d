// Circulant-embedding set-up and per-sample field generation.
//
// Set-up (Algorithm 1 steps 1-3, §2.1-2.2; Algorithm 2 step 4(b)):
//   first column c[i2][i1] = C_pad(d(i1)/n, d(i2)/n), d(i) = min(i, P-i), on
//   the device in FP64; Lambda = unnormalised +i 2D DFT of c by the library's
//   FP64 shared-memory FFT; FP64 positivity check; doubling of P while the
//   check fails; smoothing masks on the host (selection of the keep-th largest
//   eigenvalue, tie groups dropped whole); resident sqrt(Lambda~) tables.
//
// Sampling (Algorithm 1 step 4(a)-(f)), two kernels per batch:
//   row pass   : xi generated in registers (Philox), w = sqrt(Lambda~) xi,
//                real-input DFT along x of two real lines packed as one
//                complex line (two rows of w, or the fine- and coarse-masked
//                copies of one row), outputs x = 0..n kept, transposed to
//                Y[x][k2] so the column pass reads contiguous lines;
//   column pass: DFT along y, outputs y = 0..n kept, u = (Re v + Im v)/P
//                (1/sqrt(s) = 1/P), k = exp(u) written x-fastest; the plain
//                coarse field is the fine field at even vertices.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstring>
#include <vector>

#include "bulk.cuh"
#include "fft.cuh"
#include "rng.cuh"
#include "sce_internal.cuh"

using namespace sce;

// ------------------------------------------------------------------ covariance
__device__ double cov_eval(int kind, double nu, double lam, double sigma2, double t1, double t2) {
    if (kind == CE_COV_SEP_EXP) return sigma2 * exp(-(fabs(t1) + fabs(t2)) / lam);
    const double r = sqrt(t1 * t1 + t2 * t2);
    if (nu == 0.5) return sigma2 * exp(-r / lam);
    if (nu == 1.5) {
        const double z = sqrt(3.0) * r / lam;
        return sigma2 * (1.0 + z) * exp(-z);
    }
    const double z = sqrt(5.0) * r / lam;   // nu == 2.5
    return sigma2 * (1.0 + z + z * z / 3.0) * exp(-z);
}

__device__ double eta_fn(double x) { return x > 0.0 ? exp(-1.0 / x) : 0.0; }

// cutoff phi of §2.2 (1 on [-1,1], 0 outside [-kappa, kappa])
__device__ double phi_cut(double t, double kappa) {
    const double a = fabs(t);
    const double e1 = eta_fn((kappa - a) / (kappa - 1.0));
    const double e2 = eta_fn((a - 1.0) / (kappa - 1.0));
    return e1 / (e1 + e2);
}

// Eq. (2.7): sum over shifts n in {-2..2}^2 of (C phi_kappa)(x + 2 l n)
__device__ double cov_ext(int kind, double nu, double lam, double sigma2, double x1, double x2,
                          double ell) {
    const double kappa = 2.0 * ell - 1.0;
    double total = 0.0;
    for (int n1 = -2; n1 <= 2; ++n1) {
        for (int n2 = -2; n2 <= 2; ++n2) {
            const double y1 = x1 + 2.0 * ell * n1;
            const double y2 = x2 + 2.0 * ell * n2;
            const double w = phi_cut(fmax(fabs(y1), fabs(y2)), kappa);
            if (w > 0.0) total += cov_eval(kind, nu, lam, sigma2, y1, y2) * w;
        }
    }
    return total;
}

__global__ void first_column_kernel(ce_cov cov, int n, int J, int P, int mode, double2 *c) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * P) return;
    const int i1 = (int)(idx % P), i2 = (int)(idx / P);
    const double t1 = (double)min(i1, P - i1) / (double)n;
    const double t2 = (double)min(i2, P - i2) / (double)n;
    double v;
    if (mode == CE_PAD_SMOOTH)
        v = cov_ext(cov.kind, cov.nu, cov.lambda, cov.sigma2, t1, t2, 1.0 + (double)J / (double)n);
    else
        v = cov_eval(cov.kind, cov.nu, cov.lambda, cov.sigma2, t1, t2);
    c[idx] = make_double2(v, 0.0);
}

// One complex line per block, in place: data[line*line_stride + q*elem_stride].
template <int MAXB>
__global__ void fft_lines_f64_kernel(double2 *data, int logP, long long line_stride,
                                     long long elem_stride, const double2 *tw) {
    extern __shared__ double2 sm_lines[];
    const int P = 1 << logP;
    double2 *base = data + (long long)blockIdx.x * line_stride;
    for (int q = threadIdx.x; q < P; q += blockDim.x) sm_lines[fft_pad(q)] = base[q * elem_stride];
    __syncthreads();
    smem_fft<double, MAXB>(sm_lines, logP, tw, threadIdx.x, blockDim.x);
    for (int q = threadIdx.x; q < P; q += blockDim.x) base[q * elem_stride] = sm_lines[fft_pad(q)];
}

// min Re, max Re, max |Im| (one block, fixed-order tree).
__global__ void spectrum_stats_kernel(const double2 *L, long long s, double *out3) {
    __shared__ double smin[1024], smax[1024], simag[1024];
    double mn = 1e300, mx = -1e300, im = 0.0;
    for (long long i = threadIdx.x; i < s; i += blockDim.x) {
        const double2 v = L[i];
        mn = fmin(mn, v.x);
        mx = fmax(mx, v.x);
        im = fmax(im, fabs(v.y));
    }
    smin[threadIdx.x] = mn;
    smax[threadIdx.x] = mx;
    simag[threadIdx.x] = im;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + w]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
            simag[threadIdx.x] = fmax(simag[threadIdx.x], simag[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out3[0] = smin[0];
        out3[1] = smax[0];
        out3[2] = simag[0];
    }
}

__global__ void clip_real_kernel(const double2 *L, long long s, double *lam) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < s) lam[i] = fmax(L[i].x, 0.0);
}

__global__ void sqrt_table_kernel(const double *lam, const unsigned char *mask, long long s,
                                  double *sq64, float *sq32) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s) return;
    const double v = (mask == nullptr || mask[i]) ? sqrt(lam[i]) : 0.0;
    sq64[i] = v;
    sq32[i] = (float)v;
}

// Keep-mask of §2.4 / Algorithm 2 step 4(b) with the tie rule: a = keep-th
// largest, b = (keep+1)-th largest; if a - b > tol |a| keep Lambda >= a, else
// keep Lambda > a + tol |a| (the straddling tie group is dropped whole).
long long sce_keep_mask(const std::vector<double> &L, long long keep, double tol,
                        std::vector<unsigned char> &mask) {
    const long long s = (long long)L.size();
    mask.assign(s, 1);
    if (keep < 0 || keep >= s) return s;
    if (keep == 0) {
        std::fill(mask.begin(), mask.end(), 0);
        return 0;
    }
    std::vector<double> v(L);
    std::nth_element(v.begin(), v.begin() + (keep - 1), v.end(), std::greater<double>());
    const double a = v[keep - 1];
    const double b = *std::max_element(v.begin() + keep, v.end());
    const double tabs = tol * std::fabs(a);
    long long kept = 0;
    if (a - b > tabs) {
        for (long long i = 0; i < s; ++i) kept += (mask[i] = (L[i] >= a) ? 1 : 0);
    } else {
        const double thr = a + tabs;
        for (long long i = 0; i < s; ++i) kept += (mask[i] = (L[i] > thr) ? 1 : 0);
    }
    return kept;
}

static int fft2_f64(double2 *d, int P, cudaStream_t st) {
    int status = CE_OK;
    const double2 *tw = sce_twiddles64(P, &status);
    if (status != CE_OK) return status;
    const int logP = ilog2(P);
    const int nthr = std::max(1, std::min(256, P / 4));
    const size_t smem = (size_t)fft_line_pitch(P) * sizeof(double2);
    SCE_TRY(sce_raise_smem_limit((const void *)fft_lines_f64_kernel<8>, smem));
    // rows (contiguous), then columns (stride P)
    fft_lines_f64_kernel<8><<<P, nthr, smem, st>>>(d, logP, P, 1, tw);
    SCE_CUDA(cudaGetLastError());
    fft_lines_f64_kernel<8><<<P, nthr, smem, st>>>(d, logP, 1, P, tw);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

extern "C" int ce_setup_embedding(const ce_cov *cov, int n, const ce_pad *pad,
                                  const ce_smoothing *sm, void *stream, ce_embedding_t *out,
                                  ce_embedding_info *info) {
    if (!cov || !pad || !out) return CE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!is_pow2(n) || n < 4 || n > 4096) return CE_ERR_INVALID_ARG;
    if (!(cov->lambda > 0) || !(cov->sigma2 > 0)) return CE_ERR_INVALID_ARG;
    if (cov->kind == CE_COV_MATERN) {
        if (!(cov->nu == 0.5 || cov->nu == 1.5 || cov->nu == 2.5)) return CE_ERR_INVALID_ARG;
    } else if (cov->kind != CE_COV_SEP_EXP) {
        return CE_ERR_INVALID_ARG;
    }
    if (pad->mode < CE_PAD_NONE || pad->mode > CE_PAD_SMOOTH) return CE_ERR_INVALID_ARG;
    const int max_P = pad->max_P > 0 ? std::min(pad->max_P, 8192) : 8192;
    int J = pad->J >= 0 ? pad->J : (pad->mode == CE_PAD_SMOOTH ? n : 0);
    if (pad->mode == CE_PAD_SMOOTH && J < 1) return CE_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);

    double2 *Lc = nullptr;
    double *dstats = nullptr;
    int P = 0;
    double stats[3] = {0, 0, 0};
    for (;;) {
        P = 2 * (n + J);
        if (!is_pow2(P) || P < 8 || P > max_P) {
            if (Lc) sce_free(Lc, st);
            return P > max_P ? CE_ERR_NOT_PSD : CE_ERR_INVALID_ARG;
        }
        const long long s = (long long)P * P;
        if (Lc) sce_free(Lc, st);
        SCE_TRY(sce_alloc_t(&Lc, s, st));
        if (!dstats) SCE_TRY(sce_alloc_t(&dstats, 3, st));
        first_column_kernel<<<(unsigned)((s + 255) / 256), 256, 0, st>>>(*cov, n, J, P, pad->mode, Lc);
        SCE_CUDA(cudaGetLastError());
        SCE_TRY(fft2_f64(Lc, P, st));
        spectrum_stats_kernel<<<1, 1024, 0, st>>>(Lc, s, dstats);
        SCE_CUDA(cudaGetLastError());
        SCE_CUDA(cudaMemcpyAsync(stats, dstats, sizeof(stats), cudaMemcpyDeviceToHost, st));
        SCE_CUDA(cudaStreamSynchronize(st));
        if (stats[0] >= -1e-12 * stats[1]) break;
        if (pad->mode == CE_PAD_NONE || 2 * P > max_P) {
            sce_free(Lc, st);
            sce_free(dstats, st);
            cudaStreamSynchronize(st);
            return CE_ERR_NOT_PSD;
        }
        J = P - n;   // P -> 2P
    }

    ce_embedding_s *e = new ce_embedding_s();
    cudaGetDevice(&e->device);
    e->n = n;
    e->P = P;
    e->J = J;
    e->mode = pad->mode;
    e->cov = *cov;
    e->s = (long long)P * P;
    e->lambda_min = stats[0];
    e->lambda_max = stats[1];
    e->max_imag = stats[2];
    const long long s = e->s;
    int rc = CE_OK;
    auto fail = [&](int code) {
        ce_destroy(e);
        sce_free(Lc, st);
        sce_free(dstats, st);
        cudaStreamSynchronize(st);
        return code;
    };
    if (cudaMalloc(&e->lam, s * sizeof(double)) != cudaSuccess) return fail(CE_ERR_OOM);
    clip_real_kernel<<<(unsigned)((s + 255) / 256), 256, 0, st>>>(Lc, s, e->lam);
    if (cudaGetLastError() != cudaSuccess) return fail(CE_ERR_CUDA);

    // CE_KEEP_TAU_SQRT_S: drop tau = sqrt(s) = P eigenvalues (the rule of §4)
    auto resolve = [&](long long k) { return k == CE_KEEP_TAU_SQRT_S ? s - (long long)e->P : k; };
    long long keep_f = sm ? resolve(sm->keep_fine) : -1, keep_c = sm ? resolve(sm->keep_coarse) : -1;
    const double tol = (sm && sm->tie_rel_tol > 0) ? sm->tie_rel_tol : 1e-10;
    const bool need_f = keep_f >= 0 && keep_f < s;
    const bool need_c = keep_c >= 0 && keep_c < s;
    std::vector<double> hl;
    if (need_f || need_c) {
        hl.resize(s);
        if (cudaMemcpyAsync(hl.data(), e->lam, s * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(CE_ERR_CUDA);
    }
    e->keep_eff_fine = need_f ? sce_keep_mask(hl, keep_f, tol, e->mask_f) : s;
    if (need_c && need_f && keep_c == keep_f) {
        e->mask_c = e->mask_f;
        e->keep_eff_coarse = e->keep_eff_fine;
    } else {
        e->keep_eff_coarse = need_c ? sce_keep_mask(hl, keep_c, tol, e->mask_c) : s;
    }
    if (!need_f) e->mask_f.assign(s, 1);
    if (!need_c) e->mask_c.assign(s, 1);
    e->coarse_distinct = e->mask_c != e->mask_f;

    unsigned char *dmask = nullptr;
    if ((rc = sce_alloc_t(&dmask, s, st)) != CE_OK) return fail(rc);
    const unsigned blocks = (unsigned)((s + 255) / 256);
    if (cudaMalloc(&e->sq64_f, s * sizeof(double)) != cudaSuccess) return fail(CE_ERR_OOM);
    if (cudaMalloc(&e->sq32_f, s * sizeof(float)) != cudaSuccess) return fail(CE_ERR_OOM);
    if (cudaMemcpyAsync(dmask, e->mask_f.data(), s, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(CE_ERR_CUDA);
    sqrt_table_kernel<<<blocks, 256, 0, st>>>(e->lam, dmask, s, e->sq64_f, e->sq32_f);
    if (e->coarse_distinct) {
        if (cudaMalloc(&e->sq64_c, s * sizeof(double)) != cudaSuccess) return fail(CE_ERR_OOM);
        if (cudaMalloc(&e->sq32_c, s * sizeof(float)) != cudaSuccess) return fail(CE_ERR_OOM);
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CE_ERR_CUDA);
        if (cudaMemcpyAsync(dmask, e->mask_c.data(), s, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail(CE_ERR_CUDA);
        sqrt_table_kernel<<<blocks, 256, 0, st>>>(e->lam, dmask, s, e->sq64_c, e->sq32_c);
    } else {
        e->sq64_c = e->sq64_f;
        e->sq32_c = e->sq32_f;
    }
    if (cudaGetLastError() != cudaSuccess) return fail(CE_ERR_CUDA);
    sce_free(dmask, st);
    sce_free(Lc, st);
    sce_free(dstats, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        ce_destroy(e);
        return CE_ERR_CUDA;
    }
    if (info) {
        info->n = n;
        info->P = P;
        info->J = J;
        info->s = s;
        info->keep_eff_fine = e->keep_eff_fine;
        info->keep_eff_coarse = e->keep_eff_coarse;
        info->lambda_min = e->lambda_min;
        info->lambda_max = e->lambda_max;
        info->max_imag = e->max_imag;
    }
    *out = e;
    return CE_OK;
}

extern "C" void ce_destroy(ce_embedding_t e) {
    if (!e) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(e->device);
    cudaDeviceSynchronize();
    if (e->sq64_c && e->sq64_c != e->sq64_f) cudaFree(e->sq64_c);
    if (e->sq32_c && e->sq32_c != e->sq32_f) cudaFree(e->sq32_c);
    if (e->sq64_f) cudaFree(e->sq64_f);
    if (e->sq32_f) cudaFree(e->sq32_f);
    if (e->lam) cudaFree(e->lam);
    cudaSetDevice(cur);
    delete e;
}

extern "C" int ce_get_eigenvalues(ce_embedding_t e, double *dst, int dst_on_device, void *stream) {
    if (!e || !dst) return CE_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    SCE_CUDA(cudaMemcpyAsync(dst, e->lam, e->s * sizeof(double),
                             dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!dst_on_device) SCE_CUDA(cudaStreamSynchronize(st));
    return CE_OK;
}

extern "C" int ce_get_mask(ce_embedding_t e, int which, unsigned char *dst_host) {
    if (!e || !dst_host || which < 0 || which > 1) return CE_ERR_INVALID_ARG;
    const std::vector<unsigned char> &m = which == 0 ? e->mask_f : e->mask_c;
    std::memcpy(dst_host, m.data(), m.size());
    return CE_OK;
}

// ------------------------------------------------------------------ normals
template <typename R>
__global__ void normals_kernel(uint64_t seed, uint32_t level, uint64_t first_sample, int count,
                               long long len, R *out) {
    const long long nq = len / 4;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nq * count) return;
    const long long c = idx / nq, q = idx % nq;
    R z[4];
    Normals<R>::gen4(philox_block(seed, level, first_sample + (uint64_t)c, (uint32_t)q), z);
    R *o = out + c * len + 4 * q;
#pragma unroll
    for (int r = 0; r < 4; ++r) o[r] = z[r];
}

extern "C" int ce_normals(uint64_t seed, uint32_t level, uint64_t first_sample, int count,
                          long long len, int precision, void *out, void *stream) {
    if (!out || count < 0 || len < 0 || (len & 3) || len / 4 > (1LL << 32) ||
        (precision != 32 && precision != 64))
        return CE_ERR_INVALID_ARG;
    if (count == 0 || len == 0) return CE_OK;
    cudaStream_t st = as_stream(stream);
    const long long total = (len / 4) * count;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (precision == 64)
        normals_kernel<double><<<blocks, 256, 0, st>>>(seed, level, first_sample, count, len, (double *)out);
    else
        normals_kernel<float><<<blocks, 256, 0, st>>>(seed, level, first_sample, count, len, (float *)out);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

// ------------------------------------------------------------------ row pass
// Block = F lines x tpf threads.  Plain mode (sq_c == nullptr): line u packs
// rows 2u and 2u+1 as real and imaginary parts.  Masked mode: line u = row u
// with the fine-masked w as real part and the coarse-masked w as imaginary part.
// Four normals of grid indices 4q .. 4q+3 (q = g + P/4 k2): Philox (Monte
// Carlo) or the shifted lattice of point `sample` (QMC, qa.zr != nullptr).
template <typename R, bool QMC>
__device__ __forceinline__ void row_normals4(uint64_t seed, uint32_t level, uint64_t sample,
                                             uint32_t q, const QmcArgs &qa, R xi[4]) {
    if constexpr (!QMC) {
        Normals<R>::gen4(philox_block(seed, level, sample, q), xi);
    } else {
        const uint4 w = philox_block(seed, SCE_QMC_SHIFT_LEVEL, qa.shift_sample, q);
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
        const double invN = 1.0 / (double)qa.N;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t zi = (sample * (uint64_t)qa.zr[4 * (size_t)q + r]) & (uint64_t)(qa.N - 1);
            double y = (double)zi * invN + ((double)ww[r] + 0.5) * 0x1p-32;
            y -= floor(y);
            if constexpr (sizeof(R) == 8) {
                xi[r] = y < 0.5 ? normcdfinv(y) : -normcdfinv(1.0 - y);
            } else {
                xi[r] = y < 0.5 ? normcdfinvf((float)y) : -normcdfinvf((float)(1.0 - y));
            }
        }
    }
}

// The row-pass work of block (bx, sample slot sl) of a launch with F * tpf
// threads; every thread of the block calls it (it synchronises the block).
template <typename R, int MAXB, bool QMC>
__device__ __forceinline__ void ce_row_block(
    const R *__restrict__ sq_f, const R *__restrict__ sq_c, const typename C2<R>::T *__restrict__ tw,
    int P, int logP, int m, uint64_t seed, uint32_t level, uint64_t first_sample, int F, int tpf,
    typename C2<R>::T *__restrict__ Yf, typename C2<R>::T *__restrict__ Yc, const QmcArgs &qa,
    int bx, int sl, unsigned char *smem_raw) {
    using R2 = typename C2<R>::T;
    R2 *sm = reinterpret_cast<R2 *>(smem_raw);
    const uint64_t sample = first_sample + (uint64_t)sl;
    const int f = threadIdx.x / tpf, t = threadIdx.x - f * tpf;
    const bool masked = sq_c != nullptr;
    const int units = masked ? P : P / 2;
    const int u0 = bx * F;
    const int unit = u0 + f;
    const int LP = fft_line_pitch(P);
    R2 *buf = sm + (size_t)f * LP;
    const int P4 = P >> 2;
    if (unit < units) {
        if (masked) {
            const int k2 = unit;
            const R *rf = sq_f + (size_t)k2 * P;
            const R *rc = sq_c + (size_t)k2 * P;
            for (int g = t; g < P4; g += tpf) {
                R xi[4];
                row_normals4<R, QMC>(seed, level, sample, (uint32_t)(g + P4 * k2), qa, xi);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k1 = 4 * g + r;
                    buf[fft_pad(k1)] = R2{rf[k1] * xi[r], rc[k1] * xi[r]};
                }
            }
        } else {
            const int ka = 2 * unit, kb = ka + 1;
            const R *ra = sq_f + (size_t)ka * P;
            const R *rb = sq_f + (size_t)kb * P;
            for (int g = t; g < P4; g += tpf) {
                R xa[4], xb[4];
                row_normals4<R, QMC>(seed, level, sample, (uint32_t)(g + P4 * ka), qa, xa);
                row_normals4<R, QMC>(seed, level, sample, (uint32_t)(g + P4 * kb), qa, xb);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k1 = 4 * g + r;
                    buf[fft_pad(k1)] = R2{ra[k1] * xa[r], rb[k1] * xb[r]};
                }
            }
        }
    }
    __syncthreads();
    line_fft<R, MAXB>(buf, logP, tw, t, tpf);
    // split the packed transform: A = (Z[x] + conj Z[-x])/2, B = (Z[x] - conj Z[-x])/(2i)
    const R half = R(0.5);
    const int nthr = blockDim.x;
    if (!masked) {
        const int rows = 2 * F;
        const int k2base = 2 * u0;
        const long long total = (long long)(m + 1) * rows;
        for (long long idx = threadIdx.x; idx < total; idx += nthr) {
            const int x = (int)(idx / rows), rr = (int)(idx - (long long)x * rows);
            const int ff = rr >> 1;
            if (u0 + ff >= units) continue;
            const R2 *b = sm + (size_t)ff * LP;
            const R2 z = b[fft_pad(x)], zm = b[fft_pad((P - x) & (P - 1))];
            R2 o;
            if ((rr & 1) == 0) o = R2{half * (z.x + zm.x), half * (z.y - zm.y)};
            else o = R2{half * (z.y + zm.y), half * (zm.x - z.x)};
            Yf[((size_t)sl * (m + 1) + x) * P + k2base + rr] = o;
        }
    } else {
        const long long total = (long long)(m + 1) * F;
        const int mc = m / 2;
        for (long long idx = threadIdx.x; idx < total; idx += nthr) {
            const int x = (int)(idx / F), ff = (int)(idx - (long long)x * F);
            if (u0 + ff >= units) continue;
            const R2 *b = sm + (size_t)ff * LP;
            const R2 z = b[fft_pad(x)], zm = b[fft_pad((P - x) & (P - 1))];
            Yf[((size_t)sl * (m + 1) + x) * P + u0 + ff] = R2{half * (z.x + zm.x), half * (z.y - zm.y)};
            if ((x & 1) == 0)
                Yc[((size_t)sl * (mc + 1) + (x >> 1)) * P + u0 + ff] =
                    R2{half * (z.y + zm.y), half * (zm.x - z.x)};
        }
    }
}

template <typename R, int MAXB, bool QMC = false, int MINB = 4>
__global__ void __launch_bounds__(256, MINB) ce_row_kernel(
    const R *__restrict__ sq_f, const R *__restrict__ sq_c, const typename C2<R>::T *__restrict__ tw,
    int P, int logP, int m, uint64_t seed, uint32_t level, uint64_t first_sample, int F, int tpf,
    typename C2<R>::T *__restrict__ Yf, typename C2<R>::T *__restrict__ Yc, QmcArgs qa) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ce_row_block<R, MAXB, QMC>(sq_f, sq_c, tw, P, logP, m, seed, level, first_sample, F, tpf, Yf,
                               Yc, qa, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename R> __device__ __forceinline__ R exp_r(R x);
template <> __device__ __forceinline__ float exp_r<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double exp_r<double>(double x) { return exp(x); }

// ------------------------------------------------------------------ column pass
// coarse == 0: lines x = 0..m of Y (fine field), outputs y = 0..m -> kf, and
//              (kc_plain != nullptr) kc_plain at even (x, y).
// coarse == 1: lines xc = 0..m/2 of Y (coarse-masked), outputs y = 2 yc -> kout.
// The column-pass work of block (bx, sample slot sl) of a launch with F * tpf
// threads; every thread of the block calls it (it synchronises the block).
template <typename R, int MAXB>
__device__ __forceinline__ void ce_col_block(
    const typename C2<R>::T *__restrict__ Y, int ncols, int P, int logP, int m, int F, int tpf,
    const typename C2<R>::T *__restrict__ tw, int coarse, R *__restrict__ kout,
    R *__restrict__ kc_plain, int bx, int sl, unsigned char *smem_raw) {
    using R2 = typename C2<R>::T;
    R2 *sm = reinterpret_cast<R2 *>(smem_raw);
    const int f = threadIdx.x / tpf, t = threadIdx.x - f * tpf;
    const int x0 = bx * F;
    const int col = x0 + f;
    const int LP = fft_line_pitch(P);
    R2 *buf = sm + (size_t)f * LP;
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        if (tpf * 16 == P) {   // radix 16: the first pass's inputs straight into registers
            R2 v[16];
            const R2 *src = Y + ((size_t)sl * ncols + min(col, ncols - 1)) * P;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = src[t + r * tpf];
            smem_fft16_regs<R>(buf, v, logP, tw, t, tpf);
            done = true;
        }
    }
    if (!done) {
        if (col < ncols) {
            const R2 *src = Y + ((size_t)sl * ncols + col) * P;
            for (int q = t; q < P; q += tpf) buf[fft_pad(q)] = src[q];
        }
        __syncthreads();
        line_fft<R, MAXB>(buf, logP, tw, t, tpf);
    }
    const R invP = R(1) / R(P);
    const int mc = m / 2;
    const int nthr = blockDim.x;
    if (!coarse) {
        const long long total = (long long)(m + 1) * F;
        for (long long idx = threadIdx.x; idx < total; idx += nthr) {
            const int y = (int)(idx / F), ff = (int)(idx - (long long)y * F);
            const int x = x0 + ff;
            if (x >= ncols) continue;
            const R2 v = sm[(size_t)ff * LP + fft_pad(y)];
            const R k = exp_r<R>((v.x + v.y) * invP);
            kout[((size_t)sl * (m + 1) + y) * (m + 1) + x] = k;
            if (kc_plain && ((x | y) & 1) == 0)
                kc_plain[((size_t)sl * (mc + 1) + (y >> 1)) * (mc + 1) + (x >> 1)] = k;
        }
    } else {
        const long long total = (long long)(mc + 1) * F;
        for (long long idx = threadIdx.x; idx < total; idx += nthr) {
            const int yc = (int)(idx / F), ff = (int)(idx - (long long)yc * F);
            const int xc = x0 + ff;
            if (xc >= ncols) continue;
            const R2 v = sm[(size_t)ff * LP + fft_pad(2 * yc)];
            kout[((size_t)sl * (mc + 1) + yc) * (mc + 1) + xc] = exp_r<R>((v.x + v.y) * invP);
        }
    }
}

template <typename R, int MAXB, int MINB = 4>
__global__ void __launch_bounds__(256, MINB) ce_col_kernel(
    const typename C2<R>::T *__restrict__ Y, int ncols, int P, int logP, int m, int F, int tpf,
    const typename C2<R>::T *__restrict__ tw, int coarse, R *__restrict__ kout,
    R *__restrict__ kc_plain) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ce_col_block<R, MAXB>(Y, ncols, P, logP, m, F, tpf, tw, coarse, kout, kc_plain, blockIdx.x,
                          blockIdx.y, smem_raw);
}

// ------------------------------------------------------- column pass, staged
// The FP32 column pass for P = 16..2048 with its lines brought in by bulk
// copies.  Lines are numbered across the launch's samples, line l = sl *
// ncols + x, and lie one after the other in Y, so CB_G = 2048 / P consecutive
// lines are one contiguous 16 KB chunk.  A persistent block of CB_THREADS
// threads (P/16 per line, CB_G lines at once) takes chunks blockIdx.x,
// blockIdx.x + gridDim.x, ...; two stages of shared memory alternate, and the
// copy of the next chunk is in flight while the current one is transformed,
// in place: each thread reads its 16 first-pass inputs from the copied
// (unpadded) lines, and after a block barrier the radix-16 passes run on the
// same memory in the padded line layout.  The butterflies, twiddles and the
// exp epilogue are the per-block kernel's, so both give the same bits.  A
// chunk whose copy does not land within wait_cycles gets NaN outputs (and so
// does every later chunk of the block; *err is set), which the solver turns
// into CE_ERR_NONFINITE.
constexpr int CB_THREADS = 128;
constexpr int CB_ELEMS = CB_THREADS * 16;   // complex values per chunk

__host__ __device__ constexpr size_t col_bulk_stage_len(int P) {
    return (size_t)(CB_ELEMS / P) * fft_line_pitch(P);   // float2 per stage
}
__host__ __device__ constexpr size_t col_bulk_smem(int P) {
    return 2 * col_bulk_stage_len(P) * sizeof(float2) + 2 * sizeof(uint64_t);
}

template <int MINB>
__global__ void __launch_bounds__(CB_THREADS, MINB) ce_col_bulk_kernel(
    const float2 *__restrict__ Y, int nlines, int ncols, int P, int logP, int m,
    const float2 *__restrict__ tw, int coarse, float *__restrict__ kout,
    float *__restrict__ kc_plain, long long wait_cycles, int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tpf = P >> 4, G = CB_ELEMS / P, SL = (int)col_bulk_stage_len(P);
    float2 *stg = reinterpret_cast<float2 *>(smem_raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(stg + 2 * SL);
    const int nchunks = (nlines + G - 1) / G;
    const int tid = threadIdx.x, g = tid / tpf, t = tid - g * tpf;
    if (tid == 0) {
        mbar_init(bar);
        mbar_init(bar + 1);
        mbar_init_fence();
    }
    __syncthreads();
    // thread 0: copy chunk c into stage s
    auto issue = [&](int c, int s) {
        const int l0 = c * G, nl = min(G, nlines - l0);
        const uint32_t bytes = (uint32_t)nl * (uint32_t)P * (uint32_t)sizeof(float2);
        mbar_arrive_expect(bar + s, bytes);
        bulk_copy_g2s(stg + (size_t)s * SL, Y + (size_t)l0 * P, bytes, bar + s);
    };
    int c = blockIdx.x;
    bool broken = false;
    unsigned pend = 0;    // bit s: a copy into stage s not yet waited for
    int uses0 = 0, uses1 = 0;   // completed phases of the two stages' barriers
    if (c < nchunks) {
        if (tid == 0) issue(c, 0);
        pend = 1u;
    }
    const float invP = 1.0f / (float)P;
    const int mc = m / 2, nout = coarse ? mc + 1 : m + 1;
    // the outputs of a chunk are (y, line) pairs with the line fastest: since
    // G divides CB_THREADS, each thread keeps one line of every chunk
    const int gq = tid & (G - 1), ystep = CB_THREADS / G;
    for (int k = 0; c < nchunks; c += gridDim.x, ++k) {
        const int s = k & 1;
        const int cn = c + gridDim.x;
        if (!broken && cn < nchunks) {
            // stage s ^ 1 was last touched before the barrier that ended the previous chunk
            if (tid == 0) issue(cn, s ^ 1);
            pend |= 2u >> s;
        }
        const int par = (s ? uses1 : uses0) & 1;
        const bool ok = broken || mbar_wait(bar + s, (uint32_t)par, wait_cycles);
        if (__syncthreads_or(!ok)) {
            if (!broken && tid == 0) atomicExch(err, 1);
            broken = true;
        } else if (!broken) {
            pend &= ~(1u << s);
            if (s) ++uses1;
            else ++uses0;
        }
        float2 *buf = stg + (size_t)s * SL;
        const int l0 = c * G, nl = min(G, nlines - l0);
        if (!broken) {
            float2 v[16];
            const float2 *raw = buf + (size_t)g * P;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = raw[t + r * tpf];
            __syncthreads();   // every copied value read before the padded layout overwrites it
            smem_fft16_regs<float>(buf + (size_t)g * fft_line_pitch(P), v, logP, tw, t, tpf);
        }
        if (gq < nl) {
            const int l = l0 + gq, sl = l / ncols, x = l - sl * ncols;
            const float2 *line = buf + (size_t)gq * fft_line_pitch(P);
            for (int y = tid / G; y < nout; y += ystep) {
                float kv = __int_as_float(0x7fc00000);
                if (!broken) {
                    const float2 w = line[fft_pad(coarse ? 2 * y : y)];
                    kv = exp_r<float>((w.x + w.y) * invP);
                }
                if (!coarse) {
                    kout[((size_t)sl * (m + 1) + y) * (m + 1) + x] = kv;
                    if (kc_plain && ((x | y) & 1) == 0)
                        kc_plain[((size_t)sl * (mc + 1) + (y >> 1)) * (mc + 1) + (x >> 1)] = kv;
                } else {
                    kout[((size_t)sl * (mc + 1) + y) * (mc + 1) + x] = kv;
                }
            }
        }
        // stage s consumed, and this thread's stores to it ordered before the
        // bulk copy that will reuse it
        fence_proxy_async_smem();
        __syncthreads();
    }
    // a wait that gave up: give the copies still in flight a bounded chance to land
    if (broken && tid == 0) {
        if (pend & 1u) mbar_wait(bar, (uint32_t)(uses0 & 1), wait_cycles);
        if (pend & 2u) mbar_wait(bar + 1, (uint32_t)(uses1 & 1), wait_cycles);
    }
}

struct LineCfg {
    int tpf, F, maxb;
    size_t smem;
};

template <typename R>
static LineCfg line_cfg(int P, int units) {
    LineCfg c;
    c.tpf = std::max(1, std::min(256, P / 16));
    const int bpt = (P / 4 + c.tpf - 1) / c.tpf;
    c.maxb = bpt <= 4 ? 4 : 8;
    c.F = std::max(1, 256 / c.tpf);
    const size_t line = (size_t)fft_line_pitch(P) * sizeof(typename C2<R>::T);
    const size_t budget = 96 * 1024;
    while (c.F > 1 && (size_t)c.F * line > budget) c.F >>= 1;
    while (c.F > 1 && c.F / 2 >= units) c.F >>= 1;
    c.smem = (size_t)c.F * line;
    return c;
}

// FFT launch shapes chosen by ce_autotune_fft: threads per line and lines
// per block of the row pass (plain / masked) and of the column pass, per
// (P, precision).  Absent entries use line_cfg's rule.  Every shape computes
// each butterfly the same way, so a shape changes the time, never the result.
enum { TUNE_ROW_PLAIN = 0, TUNE_ROW_MASKED = 1, TUNE_COL = 2 };
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tune;   // -> (tpf, F)

template <typename R>
static bool shape_cfg(int P, int tpf, int F, LineCfg *c) {
    const int bpt = (P / 4 + tpf - 1) / tpf;
    if (tpf < 1 || tpf > 256 || F < 1 || F * tpf > 256 || bpt > 8) return false;
    c->tpf = tpf;
    c->maxb = bpt <= 4 ? 4 : 8;
    c->F = F;
    c->smem = (size_t)F * fft_line_pitch(P) * sizeof(typename C2<R>::T);
    return c->smem <= 160 * 1024;
}

template <typename R>
static LineCfg line_cfg_tuned(int P, int units, int pass) {
    LineCfg c = line_cfg<R>(P, units);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({P, (int)sizeof(R), pass});
    if (it != g_tune.end()) {
        LineCfg t;
        if (shape_cfg<R>(P, it->second.first, it->second.second, &t)) c = t;
    }
    return c;
}

// Blocks per SM the FP32 FFT passes are compiled for (64 registers at 4; 5 and
// 6 trade registers for occupancy): SCE_ROW_MINB / SCE_COL_MINB, default 4.
static int fft_minb(const char *name) {
    const char *e = getenv(name);
    const int v = e ? atoi(e) : 4;
    return (v == 5 || v == 6) ? v : 4;
}

template <typename R, int MAXB>
static int launch_row(const ce_embedding_s *e, bool masked, const typename C2<R>::T *tw,
                      uint64_t seed, uint32_t level, uint64_t first, int count,
                      typename C2<R>::T *Yf, typename C2<R>::T *Yc, const LineCfg &c,
                      cudaStream_t st, const QmcArgs *qa = nullptr) {
    const R *sqf, *sqc;
    if constexpr (sizeof(R) == 8) {
        sqf = (const R *)e->sq64_f;
        sqc = (const R *)e->sq64_c;
    } else {
        sqf = (const R *)e->sq32_f;
        sqc = (const R *)e->sq32_c;
    }
    const int units = masked ? e->P : e->P / 2;
    SCE_TRY(sce_raise_smem_limit(qa ? (const void *)ce_row_kernel<R, MAXB, true>
                                    : (const void *)ce_row_kernel<R, MAXB, false>,
                                 c.smem));
    dim3 grid((units + c.F - 1) / c.F, count);
    const int m = e->n;
    SceProf pr(KP_ROW, st,
               (double)e->s * sizeof(R) * (masked ? 2 : 1) +
                   (double)count * (m + 1) * e->P * 2 * sizeof(R) * (masked ? 1.5 : 1.0));
    const QmcArgs q = qa ? *qa : QmcArgs{nullptr, 1u, 0};
    const int minb = (sizeof(R) == 4 && MAXB == 4 && !qa) ? fft_minb("SCE_ROW_MINB") : 4;
    if (qa)
        ce_row_kernel<R, MAXB, true><<<grid, c.F * c.tpf, c.smem, st>>>(
            sqf, masked ? sqc : nullptr, tw, e->P, ilog2(e->P), e->n, seed, level, first, c.F,
            c.tpf, Yf, Yc, q);
    else if (minb == 5) {
        SCE_TRY(sce_raise_smem_limit((const void *)ce_row_kernel<R, MAXB, false, 5>, c.smem));
        ce_row_kernel<R, MAXB, false, 5><<<grid, c.F * c.tpf, c.smem, st>>>(
            sqf, masked ? sqc : nullptr, tw, e->P, ilog2(e->P), e->n, seed, level, first, c.F,
            c.tpf, Yf, Yc, q);
    } else if (minb == 6) {
        SCE_TRY(sce_raise_smem_limit((const void *)ce_row_kernel<R, MAXB, false, 6>, c.smem));
        ce_row_kernel<R, MAXB, false, 6><<<grid, c.F * c.tpf, c.smem, st>>>(
            sqf, masked ? sqc : nullptr, tw, e->P, ilog2(e->P), e->n, seed, level, first, c.F,
            c.tpf, Yf, Yc, q);
    } else
        ce_row_kernel<R, MAXB, false><<<grid, c.F * c.tpf, c.smem, st>>>(
            sqf, masked ? sqc : nullptr, tw, e->P, ilog2(e->P), e->n, seed, level, first, c.F,
            c.tpf, Yf, Yc, q);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

// The staged column pass (SCE_COL_BULK=0: the per-block kernel instead).
__device__ int g_col_bulk_err;   // set by a staged block whose copy never landed

static bool col_bulk_on() {
    const char *e = getenv("SCE_COL_BULK");
    return !(e && atoi(e) == 0);
}

// Blocks per SM the staged column pass is compiled for (SCE_COLB_MINB: 4, 5
// or 6; 6 caps it at 80 registers, with a little spilling).
static int colb_minb() {
    const char *e = getenv("SCE_COLB_MINB");
    const int v = e ? atoi(e) : 6;
    return (v == 4 || v == 5) ? v : 6;
}

template <int MINB>
static int launch_col_bulk(const ce_embedding_s *e, const float2 *Y, int ncols, int coarse,
                           const float2 *tw, int count, float *kout, float *kc_plain,
                           cudaStream_t st) {
    const int P = e->P;
    const size_t smem = col_bulk_smem(P);
    int dev = 0, sms = 0, bps = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    SCE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SCE_TRY(sce_raise_smem_limit((const void *)ce_col_bulk_kernel<MINB>, smem));
    SCE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ce_col_bulk_kernel<MINB>,
                                                           CB_THREADS, smem));
    int *err = nullptr;
    SCE_CUDA(cudaGetSymbolAddress((void **)&err, g_col_bulk_err));
    const long long nlines = (long long)count * ncols;
    if (nlines > INT32_MAX / 2) return CE_ERR_INVALID_ARG;
    const int G = CB_ELEMS / P;
    const long long nchunks = (nlines + G - 1) / G;
    const long long grid = std::min<long long>(nchunks, (long long)sms * std::max(1, bps));
    const double rows_out = coarse ? (e->n / 2 + 1) : (e->n + 1);
    SceProf pr(KP_COL, st,
               (double)count * ncols * P * 2 * sizeof(float) +
                   (double)count * ncols * rows_out * sizeof(float) * (kc_plain ? 1.25 : 1.0));
    ce_col_bulk_kernel<MINB><<<(unsigned)grid, CB_THREADS, smem, st>>>(
        Y, (int)nlines, ncols, P, ilog2(P), e->n, tw, coarse, kout, kc_plain, 1LL << 31, err);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

template <typename R, int MAXB>
static int launch_col(const ce_embedding_s *e, const typename C2<R>::T *Y, int ncols, int coarse,
                      const typename C2<R>::T *tw, int count, R *kout, R *kc_plain,
                      const LineCfg &c, cudaStream_t st) {
    // staged form: FP32, the radix-16 line shape, lines of 16..2048 values whose
    // 16 KB chunks start on 16-byte boundaries (bulk-copy alignment)
    if constexpr (sizeof(R) == 4) {
        if (col_bulk_on() && c.tpf * 16 == e->P && e->P >= 16 && e->P <= CB_ELEMS &&
            ((uintptr_t)Y & 15) == 0) {
            const int mb = colb_minb();
            if (mb == 4)
                return launch_col_bulk<4>(e, Y, ncols, coarse, tw, count, kout, kc_plain, st);
            if (mb == 5)
                return launch_col_bulk<5>(e, Y, ncols, coarse, tw, count, kout, kc_plain, st);
            return launch_col_bulk<6>(e, Y, ncols, coarse, tw, count, kout, kc_plain, st);
        }
    }
    SCE_TRY(sce_raise_smem_limit((const void *)ce_col_kernel<R, MAXB>, c.smem));
    dim3 grid((ncols + c.F - 1) / c.F, count);
    const double rows_out = coarse ? (e->n / 2 + 1) : (e->n + 1);
    SceProf pr(KP_COL, st,
               (double)count * ncols * e->P * 2 * sizeof(R) +
                   (double)count * ncols * rows_out * sizeof(R) * (kc_plain ? 1.25 : 1.0));
    const int minb = (sizeof(R) == 4 && MAXB == 4) ? fft_minb("SCE_COL_MINB") : 4;
    if (minb == 5) {
        SCE_TRY(sce_raise_smem_limit((const void *)ce_col_kernel<R, MAXB, 5>, c.smem));
        ce_col_kernel<R, MAXB, 5><<<grid, c.F * c.tpf, c.smem, st>>>(
            Y, ncols, e->P, ilog2(e->P), e->n, c.F, c.tpf, tw, coarse, kout, kc_plain);
    } else if (minb == 6) {
        SCE_TRY(sce_raise_smem_limit((const void *)ce_col_kernel<R, MAXB, 6>, c.smem));
        ce_col_kernel<R, MAXB, 6><<<grid, c.F * c.tpf, c.smem, st>>>(
            Y, ncols, e->P, ilog2(e->P), e->n, c.F, c.tpf, tw, coarse, kout, kc_plain);
    } else
        ce_col_kernel<R, MAXB><<<grid, c.F * c.tpf, c.smem, st>>>(Y, ncols, e->P, ilog2(e->P),
                                                                   e->n, c.F, c.tpf, tw, coarse,
                                                                   kout, kc_plain);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

template <typename R>
static int sample_batch_t(ce_embedding_t e, uint64_t seed, uint32_t level, uint64_t first,
                          int count, R *kf, R *kc, cudaStream_t st, const QmcArgs *qa) {
    using R2 = typename C2<R>::T;
    int status = CE_OK;
    const R2 *tw;
    if constexpr (sizeof(R) == 8) tw = sce_twiddles64(e->P, &status);
    else tw = sce_twiddles32(e->P, &status);
    if (status != CE_OK) return status;
    const int P = e->P, m = e->n, mc = m / 2;
    const bool masked = e->coarse_distinct && kc != nullptr;
    // fine field needed for kf, and (plain) for kc
    const bool need_fine = kf != nullptr || (!masked && kc != nullptr);
    // chunk so the intermediate stays below ~512 MB
    const size_t per_sample = (size_t)(m + 1) * P * sizeof(R2) + (masked ? (size_t)(mc + 1) * P * sizeof(R2) : 0);
    int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)count, (512ull << 20) / per_sample));
    chunk = std::min(chunk, 65535);
    R2 *Yf = nullptr, *Yc = nullptr;
    R *kf_tmp = nullptr;
    SCE_TRY(sce_alloc_t(&Yf, (size_t)chunk * (m + 1) * P, st));
    if (masked) SCE_TRY(sce_alloc_t(&Yc, (size_t)chunk * (mc + 1) * P, st));
    if (need_fine && kf == nullptr) SCE_TRY(sce_alloc_t(&kf_tmp, (size_t)chunk * (m + 1) * (m + 1), st));
    const LineCfg rc = line_cfg_tuned<R>(P, masked ? P : P / 2,
                                         masked ? TUNE_ROW_MASKED : TUNE_ROW_PLAIN);
    const LineCfg cc = line_cfg_tuned<R>(P, m + 1, TUNE_COL);
    const LineCfg ccc = line_cfg_tuned<R>(P, mc + 1, TUNE_COL);
    int rcode = CE_OK;
    for (int c0 = 0; c0 < count && rcode == CE_OK; c0 += chunk) {
        const int cn = std::min(chunk, count - c0);
        R *kf_c = kf ? kf + (size_t)c0 * (m + 1) * (m + 1) : kf_tmp;
        R *kc_c = kc ? kc + (size_t)c0 * (mc + 1) * (mc + 1) : nullptr;
        if (rc.maxb == 4)
            rcode = launch_row<R, 4>(e, masked, tw, seed, level, first + c0, cn, Yf, Yc, rc, st, qa);
        else
            rcode = launch_row<R, 8>(e, masked, tw, seed, level, first + c0, cn, Yf, Yc, rc, st, qa);
        if (rcode != CE_OK) break;
        if (need_fine) {
            R *kcp = masked ? nullptr : kc_c;
            if (cc.maxb == 4)
                rcode = launch_col<R, 4>(e, Yf, m + 1, 0, tw, cn, kf_c, kcp, cc, st);
            else
                rcode = launch_col<R, 8>(e, Yf, m + 1, 0, tw, cn, kf_c, kcp, cc, st);
            if (rcode != CE_OK) break;
        }
        if (masked) {
            if (ccc.maxb == 4)
                rcode = launch_col<R, 4>(e, Yc, mc + 1, 1, tw, cn, kc_c, nullptr, ccc, st);
            else
                rcode = launch_col<R, 8>(e, Yc, mc + 1, 1, tw, cn, kc_c, nullptr, ccc, st);
        }
    }
    sce_free(Yf, st);
    sce_free(Yc, st);
    sce_free(kf_tmp, st);
    return rcode;
}

// ------------------------------------------------------------------ all levels in one launch
// ce_sample_levels: the row and column passes of several levels' fields (FP32)
// in one persistent launch.  Work items -- all row blocks of all tasks, then
// all column blocks -- are claimed in order from one device counter; a
// column block of (task, sample) first waits, bounded by clock64, for the
// per-sample counter of finished row blocks.  A waiting block only depends
// on items handed out before its own, whose blocks never wait, so the
// launch cannot deadlock whatever the residency of its blocks.
constexpr int kLevelsMax = 16;

struct LevelFieldDesc {
    const float *sqf, *sqc;   // sqc: coarse-masked sqrt(Lambda~) (masked rows), else nullptr
    const float2 *tw;
    float2 *Yf, *Yc;
    float *kf, *kc;
    uint64_t first_sample;
    uint32_t level;
    int P, logP, m, count;
    int r_tpf, r_F, r_maxb, r_blocks;   // row pass, per sample
    int c_tpf, c_F, c_maxb, c_blocks;   // fine column pass, per sample
    int q_tpf, q_F, q_maxb, q_blocks;   // coarse column pass (masked), per sample
    long long row_begin, col_begin;
    int done_off, need;                 // row counters of this task start at done_off
};

struct LevelFieldArgs {
    const LevelFieldDesc *t;   // device array of ntasks descriptors
    int ntasks;
    long long rows_total, items_total;
    uint64_t seed;
    long long wait_cycles;
};

// One item of each pass, inlined with the transform length as a compile-time
// constant (the shape then needs no registers: in the stand-alone kernels it
// comes from the constant bank).
template <int LOGP>
__device__ __forceinline__ void levels_row_item_p(const LevelFieldDesc &d, uint64_t seed, int bx,
                                                  int sl, unsigned char *smem_raw) {
    constexpr int P = 1 << LOGP, TPF = P / 16 < 256 ? P / 16 : 256, F = 256 / TPF;
    const QmcArgs q0{nullptr, 1u, 0};
    ce_row_block<float, 4, false>(d.sqf, d.sqc, d.tw, P, LOGP, d.m, seed, d.level,
                                  d.first_sample, F, TPF, d.Yf, d.Yc, q0, bx, sl, smem_raw);
}

template <int LOGP>
__device__ __forceinline__ void levels_col_item_p(const LevelFieldDesc &d, int bx, int sl,
                                                  unsigned char *smem_raw) {
    constexpr int P = 1 << LOGP, TPF = P / 16 < 256 ? P / 16 : 256, F = 256 / TPF;
    const bool fine = bx < d.c_blocks;
    ce_col_block<float, 4>(fine ? d.Yf : d.Yc, fine ? d.m + 1 : d.m / 2 + 1, P, LOGP, d.m, F, TPF,
                           d.tw, fine ? 0 : 1, fine ? d.kf : d.kc,
                           fine && !d.sqc ? d.kc : nullptr, fine ? bx : bx - d.c_blocks, sl,
                           smem_raw);
}

__device__ __noinline__ void levels_row_item(const LevelFieldDesc &d, uint64_t seed, int bx, int sl,
                                             unsigned char *smem_raw) {
    switch (d.logP) {
        case 4: levels_row_item_p<4>(d, seed, bx, sl, smem_raw); break;
        case 5: levels_row_item_p<5>(d, seed, bx, sl, smem_raw); break;
        case 6: levels_row_item_p<6>(d, seed, bx, sl, smem_raw); break;
        case 7: levels_row_item_p<7>(d, seed, bx, sl, smem_raw); break;
        case 8: levels_row_item_p<8>(d, seed, bx, sl, smem_raw); break;
        case 9: levels_row_item_p<9>(d, seed, bx, sl, smem_raw); break;
        case 10: levels_row_item_p<10>(d, seed, bx, sl, smem_raw); break;
        case 11: levels_row_item_p<11>(d, seed, bx, sl, smem_raw); break;
        default: levels_row_item_p<12>(d, seed, bx, sl, smem_raw); break;
    }
}

__device__ __noinline__ void levels_col_item(const LevelFieldDesc &d, int bx, int sl,
                                             unsigned char *smem_raw) {
    switch (d.logP) {
        case 4: levels_col_item_p<4>(d, bx, sl, smem_raw); break;
        case 5: levels_col_item_p<5>(d, bx, sl, smem_raw); break;
        case 6: levels_col_item_p<6>(d, bx, sl, smem_raw); break;
        case 7: levels_col_item_p<7>(d, bx, sl, smem_raw); break;
        case 8: levels_col_item_p<8>(d, bx, sl, smem_raw); break;
        case 9: levels_col_item_p<9>(d, bx, sl, smem_raw); break;
        case 10: levels_col_item_p<10>(d, bx, sl, smem_raw); break;
        case 11: levels_col_item_p<11>(d, bx, sl, smem_raw); break;
        default: levels_col_item_p<12>(d, bx, sl, smem_raw); break;
    }
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(256, 4) ce_levels_kernel(const LevelFieldArgs a,
                                                           unsigned long long *next,
                                                           int *rowdone, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_item;
    __shared__ int s_go;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = *(volatile int *)err ? a.items_total : (long long)atomicAdd(next, 1ull);
        __syncthreads();
        const long long it = s_item;
        if (it >= a.items_total) return;
        if (it < a.rows_total) {
            int i = 0;
            while (i + 1 < a.ntasks && it >= a.t[i + 1].row_begin) ++i;
            const LevelFieldDesc &d = a.t[i];
            const long long r = it - d.row_begin;
            const int sl = (int)(r / d.r_blocks), bx = (int)(r - (long long)sl * d.r_blocks);
            levels_row_item(d, a.seed, bx, sl, smem_raw);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();   // release: this block's rows before the count
                atomicAdd(rowdone + d.done_off + sl, 1);
            }
        } else {
            int i = 0;
            while (i + 1 < a.ntasks && it >= a.t[i + 1].col_begin) ++i;
            const LevelFieldDesc &d = a.t[i];
            const int per = d.c_blocks + d.q_blocks;
            const long long c = it - d.col_begin;
            const int sl = (int)(c / per), bx = (int)(c - (long long)sl * per);
            if (threadIdx.x == 0) {
                const long long t0 = clock64();
                int ok = 1;
                while (ld_acquire_gpu(rowdone + d.done_off + sl) < d.need) {
                    if (clock64() - t0 > a.wait_cycles || *(volatile int *)err) {
                        atomicCAS(err, 0, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(128);
                }
                s_go = ok;
            }
            __syncthreads();
            if (s_go) {
                __threadfence();
                levels_col_item(d, bx, sl, smem_raw);
            }
        }
        __syncthreads();   // shared memory and s_item are reused by the next item
    }
}

// Launch shape of a pass in the persistent kernel: P/16 threads per line (as
// every FP32 shape of ce_sample_batch) and 256 threads per block, lines
// beyond the pass's count idle.
static LineCfg levels_cfg(int P) {
    LineCfg c;
    c.tpf = std::max(1, std::min(256, P / 16));
    const int bpt = (P / 4 + c.tpf - 1) / c.tpf;
    c.maxb = bpt <= 4 ? 4 : 8;
    c.F = std::max(1, 256 / c.tpf);
    c.smem = (size_t)c.F * fft_line_pitch(P) * sizeof(float2);
    return c;
}

extern "C" int ce_sample_levels(const ce_field_task *tasks, int ntasks, uint64_t seed,
                                const ce_levels_opts *opts, void *stream) {
    if (!tasks || ntasks < 1 || ntasks > kLevelsMax) return CE_ERR_INVALID_ARG;
    const cudaStream_t st = as_stream(stream);
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    LevelFieldArgs a{};
    std::vector<LevelFieldDesc> desc(ntasks);
    a.ntasks = ntasks;
    a.seed = seed;
    a.wait_cycles = (opts && opts->wait_cycles > 0) ? opts->wait_cycles : (1LL << 31);
    const int starve = opts ? opts->starve_task : -1;
    size_t ybytes = 0, smem = 0;
    long long items = 0;
    int done_total = 0;
    std::vector<size_t> yoff(ntasks), ycoff(ntasks);
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    // row items of every task, then column items of every task
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < ntasks; ++i) {
            const ce_field_task &t = tasks[i];
            const ce_embedding_s *e = t.emb;
            if (!e || e->device != dev || t.count < 0 || !t.k_fine || e->P > 4096)
                return CE_ERR_INVALID_ARG;
            LevelFieldDesc &d = desc[i];
            const bool masked = e->coarse_distinct && t.k_coarse != nullptr;
            if (pass == 0) {
                int status = CE_OK;
                d.tw = sce_twiddles32(e->P, &status);
                if (status != CE_OK) return status;
                d.sqf = e->sq32_f;
                d.sqc = masked ? e->sq32_c : nullptr;
                d.kf = (float *)t.k_fine;
                d.kc = (float *)t.k_coarse;
                d.first_sample = t.first_sample;
                d.level = t.level;
                d.P = e->P;
                d.logP = ilog2(e->P);
                d.m = e->n;
                d.count = t.count;
                const LineCfg r = levels_cfg(e->P);
                d.r_tpf = r.tpf;
                d.r_F = r.F;
                d.r_maxb = r.maxb;
                d.r_blocks = ((masked ? e->P : e->P / 2) + r.F - 1) / r.F;
                d.c_tpf = r.tpf;
                d.c_F = r.F;
                d.c_maxb = r.maxb;
                d.c_blocks = (e->n + 1 + r.F - 1) / r.F;
                d.q_tpf = r.tpf;
                d.q_F = r.F;
                d.q_maxb = r.maxb;
                d.q_blocks = masked ? (e->n / 2 + 1 + r.F - 1) / r.F : 0;
                smem = std::max(smem, r.smem);
                d.done_off = done_total;
                done_total += t.count;
                d.need = d.r_blocks + (i == starve ? 1 : 0);
                d.row_begin = items;
                items += (long long)t.count * d.r_blocks;
                yoff[i] = ybytes;
                ybytes += align((size_t)t.count * (e->n + 1) * e->P * sizeof(float2));
                ycoff[i] = ybytes;
                if (masked) ybytes += align((size_t)t.count * (e->n / 2 + 1) * e->P * sizeof(float2));
            } else {
                d.col_begin = items;
                items += (long long)t.count * (d.c_blocks + d.q_blocks);
            }
        }
        if (pass == 0) a.rows_total = items;
    }
    a.items_total = items;
    if (items == 0) return CE_OK;
    unsigned char *Y = nullptr;
    int *ctr = nullptr;   // [0..1] next (64-bit), [2] err, [3] unused, [4..] row counters
    LevelFieldDesc *dd = nullptr;
    SCE_TRY(sce_alloc((void **)&Y, std::max<size_t>(ybytes, 256), st));
    const size_t cbytes = sizeof(int) * (4 + (size_t)done_total);
    int rc = sce_alloc((void **)&ctr, cbytes, st);
    if (rc == CE_OK) rc = sce_alloc((void **)&dd, sizeof(LevelFieldDesc) * ntasks, st);
    if (rc != CE_OK) {
        sce_free(Y, st);
        sce_free(ctr, st);
        return rc;
    }
    for (int i = 0; i < ntasks; ++i) {
        desc[i].Yf = reinterpret_cast<float2 *>(Y + yoff[i]);
        desc[i].Yc = desc[i].sqc ? reinterpret_cast<float2 *>(Y + ycoff[i]) : nullptr;
    }
    a.t = dd;
    int blocks_per_sm = 0, sms = 0;
    rc = sce_raise_smem_limit((const void *)ce_levels_kernel, smem);
    // the descriptors travel with the stream (the host vector outlives the
    // copy: the call synchronises the stream before returning)
    if (rc == CE_OK &&
        (cudaMemcpyAsync(dd, desc.data(), sizeof(LevelFieldDesc) * ntasks,
                         cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemsetAsync(ctr, 0, cbytes, st) != cudaSuccess ||
         cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
         cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, ce_levels_kernel, 256,
                                                       smem) != cudaSuccess))
        rc = CE_ERR_CUDA;
    if (rc == CE_OK) {
        const long long grid = std::min<long long>(items, (long long)sms * std::max(1, blocks_per_sm));
        double bytes = 0.0;
        for (int i = 0; i < ntasks; ++i) {
            const LevelFieldDesc &d = desc[i];
            const double per = (double)(d.m + 1) * d.P * 8.0 * (d.sqc ? 1.5 : 1.0);
            bytes += (double)d.count * (2.0 * per + 4.0 * (d.m + 1) * (d.m + 1));
        }
        SceProf pr(KP_LEVELS, st, bytes);
        ce_levels_kernel<<<(unsigned)grid, 256, smem, st>>>(
            a, reinterpret_cast<unsigned long long *>(ctr), ctr + 4, ctr + 2);
        if (cudaGetLastError() != cudaSuccess) rc = CE_ERR_CUDA;
    }
    int herr = 0;
    if (rc == CE_OK && (cudaMemcpyAsync(&herr, ctr + 2, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        rc = CE_ERR_CUDA;
    if (rc != CE_OK) cudaStreamSynchronize(st);   // the pageable copy reads desc until done
    sce_free(Y, st);
    sce_free(ctr, st);
    sce_free(dd, st);
    if (rc == CE_OK && herr) {
        sce_set_last_error_text("ce_sample_levels: a column block gave up waiting for the row "
                                "blocks of its sample");
        rc = CE_ERR_TIMEOUT;
    }
    return rc;
}

int sce_sample_batch_impl(ce_embedding_t e, uint64_t seed, uint32_t level, uint64_t first_sample,
                          int count, int precision, void *k_fine, void *k_coarse, cudaStream_t st,
                          const QmcArgs *qa) {
    if (!e || count < 0 || (precision != 32 && precision != 64)) return CE_ERR_INVALID_ARG;
    if (count == 0 || (!k_fine && !k_coarse)) return CE_OK;
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    if (dev != e->device) return CE_ERR_INVALID_ARG;
    if (precision == 64)
        return sample_batch_t<double>(e, seed, level, first_sample, count, (double *)k_fine,
                                      (double *)k_coarse, st, qa);
    return sample_batch_t<float>(e, seed, level, first_sample, count, (float *)k_fine,
                                 (float *)k_coarse, st, qa);
}

extern "C" int ce_sample_batch(ce_embedding_t e, uint64_t seed, uint32_t level,
                               uint64_t first_sample, int count, int precision, void *k_fine,
                               void *k_coarse, void *stream) {
    return sce_sample_batch_impl(e, seed, level, first_sample, count, precision, k_fine, k_coarse,
                                 as_stream(stream));
}

// ------------------------------------------------------------------ no-allocation variant
// The row/column intermediate of ce_sample_batch_noalloc lives in this fixed
// device array instead of memory allocated per call.  Every device that loads
// the library reserves it until the process exits.
static constexpr size_t kStaticScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_field_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mu;
static void *g_scratch_addr[128];

// Device address of g_field_scratch on the current device, resolved once per
// device (host code must not use the symbol itself as a pointer).
static int static_scratch(void **out) {
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return CE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        SCE_CUDA(cudaGetSymbolAddress(&p, g_field_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CE_OK;
}

template <typename R>
static int sample_batch_static_t(ce_embedding_t e, uint64_t seed, uint32_t level, uint64_t first,
                                 int count, R *kf, R *kc, unsigned char *scratch,
                                 cudaStream_t st) {
    using R2 = typename C2<R>::T;
    const double2 *tw64 = nullptr;
    const float2 *tw32 = nullptr;
    SCE_TRY(sce_twiddles_lookup(e->P, &tw64, &tw32));
    const R2 *tw;
    if constexpr (sizeof(R) == 8) tw = tw64;
    else tw = tw32;
    const int P = e->P, m = e->n, mc = m / 2;
    const bool masked = e->coarse_distinct && kc != nullptr;
    const size_t yf = (size_t)(m + 1) * P * sizeof(R2);
    const size_t yc = masked ? (size_t)(mc + 1) * P * sizeof(R2) : 0;
    const size_t per_sample = ((yf + 255) & ~(size_t)255) + ((yc + 255) & ~(size_t)255);
    if (per_sample > kStaticScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "ce_sample_batch_noalloc: one sample needs %zu bytes of scratch (n=%d, P=%d, "
                 "precision %d), above the fixed %zu-byte array",
                 per_sample, m, P, (int)(8 * sizeof(R)), kStaticScratchBytes);
        sce_set_last_error_text(msg);
        return CE_ERR_INVALID_ARG;
    }
    const int chunk = (int)std::min<size_t>({(size_t)count, kStaticScratchBytes / per_sample,
                                             (size_t)65535});
    R2 *Yf = reinterpret_cast<R2 *>(scratch);
    R2 *Yc = masked ? reinterpret_cast<R2 *>(scratch + (((size_t)chunk * yf + 255) & ~(size_t)255))
                    : nullptr;
    // the launch shapes ce_autotune_fft chose, as ce_sample_batch uses them
    // (a map lookup under a mutex; no allocation)
    const LineCfg rc = line_cfg_tuned<R>(P, masked ? P : P / 2,
                                         masked ? TUNE_ROW_MASKED : TUNE_ROW_PLAIN);
    const LineCfg cc = line_cfg_tuned<R>(P, m + 1, TUNE_COL);
    const LineCfg ccc = line_cfg_tuned<R>(P, mc + 1, TUNE_COL);
    int rcode = CE_OK;
    for (int c0 = 0; c0 < count && rcode == CE_OK; c0 += chunk) {
        const int cn = std::min(chunk, count - c0);
        R *kf_c = kf + (size_t)c0 * (m + 1) * (m + 1);
        R *kc_c = kc ? kc + (size_t)c0 * (mc + 1) * (mc + 1) : nullptr;
        if (rc.maxb == 4)
            rcode = launch_row<R, 4>(e, masked, tw, seed, level, first + c0, cn, Yf, Yc, rc, st);
        else
            rcode = launch_row<R, 8>(e, masked, tw, seed, level, first + c0, cn, Yf, Yc, rc, st);
        if (rcode != CE_OK) break;
        R *kcp = masked ? nullptr : kc_c;
        if (cc.maxb == 4)
            rcode = launch_col<R, 4>(e, Yf, m + 1, 0, tw, cn, kf_c, kcp, cc, st);
        else
            rcode = launch_col<R, 8>(e, Yf, m + 1, 0, tw, cn, kf_c, kcp, cc, st);
        if (rcode != CE_OK) break;
        if (masked) {
            if (ccc.maxb == 4)
                rcode = launch_col<R, 4>(e, Yc, mc + 1, 1, tw, cn, kc_c, nullptr, ccc, st);
            else
                rcode = launch_col<R, 8>(e, Yc, mc + 1, 1, tw, cn, kc_c, nullptr, ccc, st);
        }
    }
    return rcode;
}

extern "C" int ce_sample_batch_noalloc(ce_embedding_t e, uint64_t seed, uint32_t level,
                                       uint64_t first_sample, int count, int precision,
                                       void *k_fine, void *k_coarse, void *stream) {
    if (!e || count < 0 || (precision != 32 && precision != 64) || !k_fine)
        return CE_ERR_INVALID_ARG;
    if (count == 0) return CE_OK;
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    if (dev != e->device) return CE_ERR_INVALID_ARG;
    void *scratch = nullptr;
    SCE_TRY(static_scratch(&scratch));
    cudaStream_t st = as_stream(stream);
    if (precision == 64)
        return sample_batch_static_t<double>(e, seed, level, first_sample, count,
                                             (double *)k_fine, (double *)k_coarse,
                                             (unsigned char *)scratch, st);
    return sample_batch_static_t<float>(e, seed, level, first_sample, count, (float *)k_fine,
                                        (float *)k_coarse, (unsigned char *)scratch, st);
}

// ------------------------------------------------------------------ quasi-Monte Carlo sampler
extern "C" int ce_qmc_setup(ce_embedding_t e, uint32_t N, uint32_t a, ce_qmc_t *out) {
    if (!e || !out || N == 0 || (N & (N - 1)) != 0 || N > (1u << 31) || (a & 1u) == 0)
        return CE_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    if (dev != e->device) return CE_ERR_INVALID_ARG;
    const size_t s = (size_t)e->s;
    const int P = e->P;
    // lattice dimensions by increasing wavenumber d(k1)^2 + d(k2)^2, d(k) =
    // min(k, P - k), ties by grid index j = k1 + P k2 (an exact integer order)
    std::vector<uint32_t> order(s);
    std::vector<uint64_t> key(s);
    for (size_t j = 0; j < s; ++j) {
        const uint64_t k1 = j % P, k2 = j / P;
        const uint64_t d1 = std::min<uint64_t>(k1, P - k1), d2 = std::min<uint64_t>(k2, P - k2);
        key[j] = d1 * d1 + d2 * d2;
        order[j] = (uint32_t)j;
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return key[x] < key[y]; });
    // Korobov vector z_r = a^r mod N, placed at the grid index of rank r
    std::vector<uint32_t> zr(s);
    uint64_t z = 1 % N;
    for (size_t r = 0; r < s; ++r) {
        zr[order[r]] = (uint32_t)z;
        z = (z * a) % N;
    }
    ce_qmc_s *q = new (std::nothrow) ce_qmc_s{e, N, a, nullptr, dev};
    if (!q) return CE_ERR_OOM;
    if (cudaMalloc(&q->zr, s * sizeof(uint32_t)) != cudaSuccess) {
        delete q;
        return CE_ERR_OOM;
    }
    if (cudaMemcpy(q->zr, zr.data(), s * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(q->zr);
        delete q;
        return CE_ERR_CUDA;
    }
    *out = q;
    return CE_OK;
}

extern "C" void ce_qmc_destroy(ce_qmc_t q) {
    if (!q) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(q->device);
    cudaDeviceSynchronize();
    cudaFree(q->zr);
    cudaSetDevice(cur);
    delete q;
}

extern "C" int ce_sample_batch_qmc(ce_qmc_t q, uint64_t seed, uint32_t level, uint32_t shift,
                                   uint32_t first_point, int count, int precision, void *k_fine,
                                   void *k_coarse, void *stream) {
    if (!q || count < 0 || (uint64_t)first_point + (uint64_t)count > q->N) return CE_ERR_INVALID_ARG;
    const QmcArgs qa{q->zr, q->N, ((uint64_t)level << 32) | shift};
    return sce_sample_batch_impl(q->e, seed, level, first_point, count, precision, k_fine,
                                 k_coarse, as_stream(stream), &qa);
}

// ------------------------------------------------------------------ FFT autotuner
// Times ce_sample_batch of `count` samples of handle e for every admissible
// shape of the row pass (with the column pass at its current shape), keeps
// the fastest, then does the same for the column pass.
extern "C" int ce_autotune_fft(ce_embedding_t e, int precision, int count, int reps,
                               void *stream, int *row_tpf, int *row_F, int *col_tpf, int *col_F) {
    if (!e || count < 1 || reps < 1 || (precision != 32 && precision != 64))
        return CE_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    const int P = e->P, m = e->n, mc = m / 2;
    const size_t es = precision == 64 ? sizeof(double) : sizeof(float);
    const bool masked = e->coarse_distinct;
    void *kf = nullptr, *kc = nullptr;
    SCE_TRY(sce_alloc(&kf, (size_t)count * (m + 1) * (m + 1) * es, st));
    if (sce_alloc(&kc, (size_t)count * (mc + 1) * (mc + 1) * es, st) != CE_OK) {
        sce_free(kf, st);
        return CE_ERR_OOM;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int row_pass = masked ? TUNE_ROW_MASKED : TUNE_ROW_PLAIN;
    int rc = CE_OK;
    auto time_it = [&](float *ms) {
        for (int w = 0; w < 2 && rc == CE_OK; ++w)   // warm-up (also loads the kernels)
            rc = sce_sample_batch_impl(e, 1, 0, 0, count, precision, kf, kc, st);
        if (rc != CE_OK) return;
        cudaEventRecord(a, st);
        for (int r = 0; r < reps && rc == CE_OK; ++r)
            rc = sce_sample_batch_impl(e, 1, 0, 0, count, precision, kf, kc, st);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) rc = CE_ERR_CUDA;
        cudaEventElapsedTime(ms, a, b);
    };
    for (int pass : {row_pass, (int)TUNE_COL}) {
        const std::tuple<int, int, int> key{P, (int)es, pass};
        float best = 1e30f;
        std::pair<int, int> best_shape{0, 0};
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) best_shape = it->second;
        }
        // FP32 lines run the radix-16 FFT at P/16 threads per line (other
        // thread counts would take the radix-4 form, with other rounding)
        const std::vector<int> divs = es == 4 ? std::vector<int>{16} : std::vector<int>{32, 16, 8, 4};
        for (int div : divs) {
            const int tpf = std::max(1, P / div);
            for (int fdiv : {1, 2, 4}) {
                const int F = std::max(1, 256 / tpf / fdiv);
                LineCfg c;
                const bool ok = es == 8 ? shape_cfg<double>(P, tpf, F, &c)
                                        : shape_cfg<float>(P, tpf, F, &c);
                if (!ok) continue;
                {
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    g_tune[key] = {tpf, F};
                }
                float ms = 0.f;
                time_it(&ms);
                if (rc != CE_OK) break;
                if (ms < best) {
                    best = ms;
                    best_shape = {tpf, F};
                }
            }
            if (rc != CE_OK) break;
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (best_shape.first > 0) g_tune[key] = best_shape;
        else g_tune.erase(key);
        if (rc != CE_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    sce_free(kf, st);
    sce_free(kc, st);
    if (rc != CE_OK) return rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto get = [&](int pass, int *tpf, int *F) {
        auto it = g_tune.find({P, (int)es, pass});
        if (tpf) *tpf = it != g_tune.end() ? it->second.first : 0;
        if (F) *F = it != g_tune.end() ? it->second.second : 0;
    };
    get(row_pass, row_tpf, row_F);
    get(TUNE_COL, col_tpf, col_F);
    return CE_OK;
}

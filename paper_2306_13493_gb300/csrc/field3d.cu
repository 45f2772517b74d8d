// Circulant embedding and field generation on three-dimensional grids
// (§2.1-2.2 in d = 3; the paper states the construction for d = 1, 2 and
// says higher dimensions follow the same pattern; Eq. (2.7) and the smoothing
// of §2.4 are written for general d).
//
// Grid (n+1)^3, vertex (i1, i2, i3) at index i1 + (n+1) i2 + (n+1)^2 i3;
// embedding P^3, s = P^3, array index k1 + P k2 + P^2 k3.
//
// Set-up: first column c = C_pad(d(k1)/n, d(k2)/n, d(k3)/n) in FP64 (C_ext
// sums the 5^3 shifts of Eq. (2.7)), Lambda = threefold unnormalised +i DFT
// by FP64 shared-memory line FFTs along the three axes, positivity check,
// doubling of P, smoothing masks on the host, resident FP32 sqrt(Lambda~).
//
// Sampling (FP32), three line passes per batch, each keeping only the
// outputs the grid needs (a pruned transform: n+1 of P outputs per axis):
//   x pass : xi generated in registers (Philox), w = sqrt(Lambda~) xi, two
//            real x-lines packed as one complex line (rows k2, k2+1, or the
//            fine- and coarse-masked copies of one row), DFT, split, keep
//            x = 0..n -> Y1[s][k3][x][k2];
//   y pass : DFT of the complex y-lines of Y1, keep y = 0..n -> Y2[s][y][x][k3];
//   z pass : DFT of the z-lines of Y2, keep z = 0..n, u = (Re v + Im v)/P^(3/2),
//            k = exp(u) written x-fastest (and the plain coarse field at even
//            vertices).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fft.cuh"
#include "rng.cuh"
#include "sce_internal.cuh"

using namespace sce;

struct ce3_embedding_s {
    int device;
    int n, P, J, mode;
    ce_cov cov;
    long long s;   // P^3
    long long keep_eff_fine, keep_eff_coarse;
    bool coarse_distinct;
    double lambda_min, lambda_max, max_imag;
    double *lam;            // P^3 eigenvalues (clipped), device
    float *sq_f, *sq_c;     // P^3 sqrt(Lambda~) fine / coarse (sq_c == sq_f unless distinct)
    std::vector<unsigned char> mask_f, mask_c;
};

namespace {

constexpr int kMaxP3 = 512;

// ------------------------------------------------------------------ covariance
__device__ double cov3_eval(int kind, double nu, double lam, double sigma2, double t1, double t2,
                            double t3) {
    if (kind == CE_COV_SEP_EXP) return sigma2 * exp(-(fabs(t1) + fabs(t2) + fabs(t3)) / lam);
    const double r = sqrt(t1 * t1 + t2 * t2 + t3 * t3);
    if (nu == 0.5) return sigma2 * exp(-r / lam);
    if (nu == 1.5) {
        const double z = sqrt(3.0) * r / lam;
        return sigma2 * (1.0 + z) * exp(-z);
    }
    const double z = sqrt(5.0) * r / lam;   // nu == 2.5
    return sigma2 * (1.0 + z + z * z / 3.0) * exp(-z);
}

__device__ double eta3(double x) { return x > 0.0 ? exp(-1.0 / x) : 0.0; }

// cutoff of §2.2: 1 on [-1, 1], 0 outside [-kappa, kappa]
__device__ double phi3(double t, double kappa) {
    const double a = fabs(t);
    const double e1 = eta3((kappa - a) / (kappa - 1.0));
    const double e2 = eta3((a - 1.0) / (kappa - 1.0));
    return e1 / (e1 + e2);
}

// Eq. (2.7) in d = 3: sum over n in {-2..2}^3 of (C phi_kappa)(x + 2 l n)
__device__ double cov3_ext(int kind, double nu, double lam, double sigma2, double x1, double x2,
                           double x3, double ell) {
    const double kappa = 2.0 * ell - 1.0;
    double total = 0.0;
    for (int n1 = -2; n1 <= 2; ++n1)
        for (int n2 = -2; n2 <= 2; ++n2)
            for (int n3 = -2; n3 <= 2; ++n3) {
                const double y1 = x1 + 2.0 * ell * n1;
                const double y2 = x2 + 2.0 * ell * n2;
                const double y3 = x3 + 2.0 * ell * n3;
                const double w = phi3(fmax(fmax(fabs(y1), fabs(y2)), fabs(y3)), kappa);
                if (w > 0.0) total += cov3_eval(kind, nu, lam, sigma2, y1, y2, y3) * w;
            }
    return total;
}

__global__ void first_column3_kernel(ce_cov cov, int n, int J, int P, int mode, double2 *c) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long s = (long long)P * P * P;
    if (idx >= s) return;
    const int i1 = (int)(idx % P);
    const int i2 = (int)((idx / P) % P);
    const int i3 = (int)(idx / ((long long)P * P));
    const double t1 = (double)min(i1, P - i1) / (double)n;
    const double t2 = (double)min(i2, P - i2) / (double)n;
    const double t3 = (double)min(i3, P - i3) / (double)n;
    double v;
    if (mode == CE_PAD_SMOOTH)
        v = cov3_ext(cov.kind, cov.nu, cov.lambda, cov.sigma2, t1, t2, t3,
                     1.0 + (double)J / (double)n);
    else
        v = cov3_eval(cov.kind, cov.nu, cov.lambda, cov.sigma2, t1, t2, t3);
    c[idx] = make_double2(v, 0.0);
}

// One FP64 line of the P^3 array per block, in place: line l starts at
// (l mod P) sa + (l div P) sb, element q at + q es.
__global__ void fft3_lines_f64_kernel(double2 *data, int logP, long long sa, long long sb,
                                      long long es, const double2 *tw) {
    extern __shared__ __align__(16) unsigned char smem_setup3[];
    double2 *sm = reinterpret_cast<double2 *>(smem_setup3);
    const int P = 1 << logP;
    const long long l = blockIdx.x;
    double2 *base = data + (l % P) * sa + (l / P) * sb;
    for (int q = threadIdx.x; q < P; q += blockDim.x) sm[fft_pad(q)] = base[q * es];
    __syncthreads();
    smem_fft<double, 4>(sm, logP, tw, threadIdx.x, blockDim.x);
    for (int q = threadIdx.x; q < P; q += blockDim.x) base[q * es] = sm[fft_pad(q)];
}

// min Re, max Re, max |Im| (one block, fixed-order tree)
__global__ void spectrum3_stats_kernel(const double2 *L, long long s, double *out3) {
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

__global__ void clip3_kernel(const double2 *L, long long s, double *lam) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < s) lam[i] = fmax(L[i].x, 0.0);
}

__global__ void sqrt3_table_kernel(const double *lam, const unsigned char *mask, long long s,
                                   float *sq) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < s) sq[i] = (float)((mask == nullptr || mask[i]) ? sqrt(lam[i]) : 0.0);
}

static int fft3_f64(double2 *d, int P, cudaStream_t st) {
    int status = CE_OK;
    const double2 *tw = sce_twiddles64(P, &status);
    if (status != CE_OK) return status;
    const int logP = ilog2(P);
    const int nthr = std::max(1, std::min(256, P / 4));
    const size_t smem = (size_t)fft_line_pitch(P) * sizeof(double2);
    SCE_TRY(sce_raise_smem_limit((const void *)fft3_lines_f64_kernel, smem));
    const long long P2 = (long long)P * P;
    fft3_lines_f64_kernel<<<(unsigned)P2, nthr, smem, st>>>(d, logP, P, P2, 1, tw);    // x
    SCE_CUDA(cudaGetLastError());
    fft3_lines_f64_kernel<<<(unsigned)P2, nthr, smem, st>>>(d, logP, 1, P2, P, tw);    // y
    SCE_CUDA(cudaGetLastError());
    fft3_lines_f64_kernel<<<(unsigned)P2, nthr, smem, st>>>(d, logP, 1, P, P2, tw);    // z
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

// ------------------------------------------------------------------ x pass
// Block = F lines x tpf threads; grid (samples, line groups): consecutive
// blocks are the same lines of consecutive samples, so each tile of the
// sqrt(Lambda~) table is read from HBM once per batch and from L2 after.
// Plain mode (sq_c == nullptr): line u packs rows 2u, 2u+1 (row = k2 + P k3)
// as real and imaginary parts.  Masked mode: line u = row u, fine-masked w
// real, coarse-masked w imaginary.  Four normals 4g..4g+3 of a row come from
// Philox block g + (P/4) row (normal j = k1 + P row).
template <int MAXB>
__global__ void __launch_bounds__(256) ce3_x_kernel(
    const float *__restrict__ sq_f, const float *__restrict__ sq_c,
    const float2 *__restrict__ tw, int P, int logP, int m, uint64_t seed, uint32_t level,
    uint64_t first_sample, int F, int tpf, float2 *__restrict__ Yf, float2 *__restrict__ Yc) {
    extern __shared__ __align__(16) unsigned char smem_x3[];
    float2 *sm = reinterpret_cast<float2 *>(smem_x3);
    const int sl = blockIdx.x;
    const uint64_t sample = first_sample + (uint64_t)sl;
    const int f = threadIdx.x / tpf, t = threadIdx.x - f * tpf;
    const bool masked = sq_c != nullptr;
    const long long units = masked ? (long long)P * P : (long long)P * P / 2;
    const long long u0 = (long long)blockIdx.y * F;
    const long long unit = u0 + f;
    const int LP = fft_line_pitch(P);
    float2 *buf = sm + (size_t)f * LP;
    const int P4 = P >> 2;
    if (unit < units) {
        if (masked) {
            const float *rf = sq_f + unit * P, *rc = sq_c + unit * P;
            for (int g = t; g < P4; g += tpf) {
                float xi[4];
                Normals<float>::gen4(philox_block(seed, level, sample, (uint32_t)(g + P4 * unit)),
                                     xi);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k1 = 4 * g + r;
                    buf[fft_pad(k1)] = float2{rf[k1] * xi[r], rc[k1] * xi[r]};
                }
            }
        } else {
            const long long ra = 2 * unit, rb = ra + 1;
            const float *pa = sq_f + ra * P, *pb = sq_f + rb * P;
            for (int g = t; g < P4; g += tpf) {
                float xa[4], xb[4];
                Normals<float>::gen4(philox_block(seed, level, sample, (uint32_t)(g + P4 * ra)), xa);
                Normals<float>::gen4(philox_block(seed, level, sample, (uint32_t)(g + P4 * rb)), xb);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k1 = 4 * g + r;
                    buf[fft_pad(k1)] = float2{pa[k1] * xa[r], pb[k1] * xb[r]};
                }
            }
        }
    }
    __syncthreads();
    line_fft<float, MAXB>(buf, logP, tw, t, tpf);
    // split the packed transform: A = (Z[x] + conj Z[-x])/2, B = (Z[x] - conj Z[-x])/(2i)
    const float half = 0.5f;
    const int nthr = blockDim.x;
    if (!masked) {
        const int rows = 2 * F;
        const long long total = (long long)(m + 1) * rows;
        for (long long idx = threadIdx.x; idx < total; idx += nthr) {
            const int x = (int)(idx / rows), rr = (int)(idx - (long long)x * rows);
            const int ff = rr >> 1;
            const long long un = u0 + ff;
            if (un >= units) continue;
            const long long row = 2 * un + (rr & 1);
            const long long k3 = row / P;
            const long long k2 = row - k3 * P;
            const float2 *b = sm + (size_t)ff * LP;
            const float2 z = b[fft_pad(x)], zm = b[fft_pad((P - x) & (P - 1))];
            float2 o;
            if ((rr & 1) == 0) o = float2{half * (z.x + zm.x), half * (z.y - zm.y)};
            else o = float2{half * (z.y + zm.y), half * (zm.x - z.x)};
            Yf[(((size_t)sl * P + k3) * (m + 1) + x) * P + k2] = o;
        }
    } else {
        const int mc = m / 2;
        const long long total = (long long)(m + 1) * F;
        for (long long idx = threadIdx.x; idx < total; idx += nthr) {
            const int x = (int)(idx / F), ff = (int)(idx - (long long)x * F);
            const long long row = u0 + ff;
            if (row >= units) continue;
            const long long k3 = row / P;
            const long long k2 = row - k3 * P;
            const float2 *b = sm + (size_t)ff * LP;
            const float2 z = b[fft_pad(x)], zm = b[fft_pad((P - x) & (P - 1))];
            Yf[(((size_t)sl * P + k3) * (m + 1) + x) * P + k2] =
                float2{half * (z.x + zm.x), half * (z.y - zm.y)};
            if ((x & 1) == 0)
                Yc[(((size_t)sl * P + k3) * (mc + 1) + (x >> 1)) * P + k2] =
                    float2{half * (z.y + zm.y), half * (zm.x - z.x)};
        }
    }
}

// ------------------------------------------------------------------ y pass
// Lines (sample, k3, x), x < nx, of Yin[s][k3][x][k2]; DFT over k2; outputs
// y = yo ystep, yo < ny, to Yout[s][yo][x][k3].  Block = F lines with
// consecutive k3 at one x (F divides P), so each output run is F values.
template <int MAXB>
__global__ void __launch_bounds__(256) ce3_y_kernel(const float2 *__restrict__ Yin, int nx, int P,
                                                    int logP, int ny, int ystep, int F, int tpf,
                                                    const float2 *__restrict__ tw,
                                                    float2 *__restrict__ Yout) {
    extern __shared__ __align__(16) unsigned char smem_y3[];
    float2 *sm = reinterpret_cast<float2 *>(smem_y3);
    const int sl = blockIdx.y;
    const int groups = P / F;
    const int x = blockIdx.x / groups, k30 = (blockIdx.x - x * groups) * F;
    const int f = threadIdx.x / tpf, t = threadIdx.x - f * tpf;
    const int LP = fft_line_pitch(P);
    float2 *buf = sm + (size_t)f * LP;
    const float2 *src = Yin + (((size_t)sl * P + k30 + f) * nx + x) * P;
    if (tpf * 16 == P) {   // radix 16: the first pass's inputs straight into registers
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = src[t + r * tpf];
        smem_fft16_regs<float>(buf, v, logP, tw, t, tpf);
    } else {
        for (int q = t; q < P; q += tpf) buf[fft_pad(q)] = src[q];
        __syncthreads();
        line_fft<float, MAXB>(buf, logP, tw, t, tpf);
    }
    const int total = ny * F;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int yo = idx / F, ff = idx - yo * F;
        Yout[(((size_t)sl * ny + yo) * nx + x) * P + k30 + ff] = sm[(size_t)ff * LP + fft_pad(yo * ystep)];
    }
}

// ------------------------------------------------------------------ z pass
// Lines (sample, yo, x), x < nx, yo < ny, of Yin[s][yo][x][k3]; DFT over k3;
// outputs z = zo zstep, zo < nz: kout[s][zo][yo][x] = exp((Re + Im) invs).
// kc_plain (fine pass only): the field at even (x, yo, zo) to the
// (mc+1)^3 coarse grid.  Block = F lines with consecutive x at one yo.
template <int MAXB>
__global__ void __launch_bounds__(256) ce3_z_kernel(const float2 *__restrict__ Yin, int nx, int ny,
                                                    int P, int logP, int nz, int zstep, int F,
                                                    int tpf, const float2 *__restrict__ tw,
                                                    float invs, float *__restrict__ kout,
                                                    float *__restrict__ kc_plain, int mc) {
    extern __shared__ __align__(16) unsigned char smem_z3[];
    float2 *sm = reinterpret_cast<float2 *>(smem_z3);
    const int sl = blockIdx.y;
    const int gx = (nx + F - 1) / F;
    const int yo = blockIdx.x / gx, x0 = (blockIdx.x - yo * gx) * F;
    const int f = threadIdx.x / tpf, t = threadIdx.x - f * tpf;
    const int LP = fft_line_pitch(P);
    float2 *buf = sm + (size_t)f * LP;
    if (tpf * 16 == P) {   // radix 16: the first pass's inputs straight into registers
        float2 v[16];
        const float2 *src = Yin + (((size_t)sl * ny + yo) * nx + min(x0 + f, nx - 1)) * P;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = src[t + r * tpf];
        smem_fft16_regs<float>(buf, v, logP, tw, t, tpf);
    } else {
        if (x0 + f < nx) {
            const float2 *src = Yin + (((size_t)sl * ny + yo) * nx + x0 + f) * P;
            for (int q = t; q < P; q += tpf) buf[fft_pad(q)] = src[q];
        }
        __syncthreads();
        line_fft<float, MAXB>(buf, logP, tw, t, tpf);
    }
    const int total = nz * F;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int zo = idx / F, ff = idx - zo * F;
        const int x = x0 + ff;
        if (x >= nx) continue;
        const float2 v = sm[(size_t)ff * LP + fft_pad(zo * zstep)];
        const float k = expf((v.x + v.y) * invs);
        kout[(((size_t)sl * nz + zo) * ny + yo) * nx + x] = k;
        if (kc_plain && ((x | yo | zo) & 1) == 0)
            kc_plain[(((size_t)sl * (mc + 1) + (zo >> 1)) * (mc + 1) + (yo >> 1)) * (mc + 1) +
                     (x >> 1)] = k;
    }
}

struct Cfg3 {
    int tpf, F, maxb;
    size_t smem;
};

// threads per line P/16 (1..256), lines per block up to 256/tpf within a
// 96 KB shared budget, at most `lines` (a power of two dividing P or P^2)
static Cfg3 cfg3(int P, long long lines) {
    Cfg3 c;
    c.tpf = std::max(1, std::min(256, P / 16));
    const int bpt = (P / 4 + c.tpf - 1) / c.tpf;
    c.maxb = bpt <= 4 ? 4 : 8;
    c.F = std::max(1, 256 / c.tpf);
    const size_t line = (size_t)fft_line_pitch(P) * sizeof(float2);
    while (c.F > 1 && (size_t)c.F * line > 96 * 1024) c.F >>= 1;
    while (c.F > 1 && c.F > lines) c.F >>= 1;
    c.smem = (size_t)c.F * line;
    return c;
}

template <int MAXB>
static int launch_x3(const ce3_embedding_s *e, bool masked, const float2 *tw, uint64_t seed,
                     uint32_t level, uint64_t first, int count, float2 *Yf, float2 *Yc,
                     const Cfg3 &c, cudaStream_t st) {
    const int P = e->P, m = e->n;
    const long long units = masked ? (long long)P * P : (long long)P * P / 2;
    SCE_TRY(sce_raise_smem_limit((const void *)ce3_x_kernel<MAXB>, c.smem));
    dim3 grid(count, (unsigned)(units / c.F));
    SceProf pr(KP_X3, st,
               (double)e->s * 4.0 * (masked ? 2 : 1) +
                   (double)count * (m + 1) * P * P * 8.0 * (masked ? 1.5 : 1.0));
    ce3_x_kernel<MAXB><<<grid, c.F * c.tpf, c.smem, st>>>(e->sq_f, masked ? e->sq_c : nullptr, tw,
                                                          P, ilog2(P), m, seed, level, first, c.F,
                                                          c.tpf, Yf, Yc);
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

static int launch_y3(const float2 *Yin, int nx, int P, int ny, int ystep, const float2 *tw,
                     int count, float2 *Yout, cudaStream_t st) {
    const Cfg3 c = cfg3(P, P);
    dim3 grid((unsigned)(nx * (P / c.F)), count);
    SceProf pr(KP_Y3, st, (double)count * nx * P * (double)(P + ny) * 8.0);
    if (c.maxb == 4) {
        SCE_TRY(sce_raise_smem_limit((const void *)ce3_y_kernel<4>, c.smem));
        ce3_y_kernel<4><<<grid, c.F * c.tpf, c.smem, st>>>(Yin, nx, P, ilog2(P), ny, ystep, c.F,
                                                           c.tpf, tw, Yout);
    } else {
        SCE_TRY(sce_raise_smem_limit((const void *)ce3_y_kernel<8>, c.smem));
        ce3_y_kernel<8><<<grid, c.F * c.tpf, c.smem, st>>>(Yin, nx, P, ilog2(P), ny, ystep, c.F,
                                                           c.tpf, tw, Yout);
    }
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

static int launch_z3(const float2 *Yin, int nx, int ny, int P, int nz, int zstep,
                     const float2 *tw, int count, float *kout, float *kc_plain, int mc,
                     cudaStream_t st) {
    const Cfg3 c = cfg3(P, nx);
    const int gx = (nx + c.F - 1) / c.F;
    dim3 grid((unsigned)(ny * gx), count);
    const float invs = (float)(1.0 / ((double)P * std::sqrt((double)P)));
    SceProf pr(KP_Z3, st,
               (double)count * nx * ny * ((double)P * 8.0 + nz * 4.0 * (kc_plain ? 1.125 : 1.0)));
    if (c.maxb == 4) {
        SCE_TRY(sce_raise_smem_limit((const void *)ce3_z_kernel<4>, c.smem));
        ce3_z_kernel<4><<<grid, c.F * c.tpf, c.smem, st>>>(Yin, nx, ny, P, ilog2(P), nz, zstep,
                                                           c.F, c.tpf, tw, invs, kout, kc_plain,
                                                           mc);
    } else {
        SCE_TRY(sce_raise_smem_limit((const void *)ce3_z_kernel<8>, c.smem));
        ce3_z_kernel<8><<<grid, c.F * c.tpf, c.smem, st>>>(Yin, nx, ny, P, ilog2(P), nz, zstep,
                                                           c.F, c.tpf, tw, invs, kout, kc_plain,
                                                           mc);
    }
    SCE_CUDA(cudaGetLastError());
    return CE_OK;
}

}  // namespace

extern "C" void ce3_destroy(ce3_embedding_t e) {
    if (!e) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(e->device);
    cudaDeviceSynchronize();
    if (e->sq_c && e->sq_c != e->sq_f) cudaFree(e->sq_c);
    if (e->sq_f) cudaFree(e->sq_f);
    if (e->lam) cudaFree(e->lam);
    cudaSetDevice(cur);
    delete e;
}

extern "C" int ce3_setup_embedding(const ce_cov *cov, int n, const ce_pad *pad,
                                   const ce_smoothing *sm, void *stream, ce3_embedding_t *out,
                                   ce_embedding_info *info) {
    if (!cov || !pad || !out) return CE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!is_pow2(n) || n < 2 || n > 256) return CE_ERR_INVALID_ARG;
    if (!(cov->lambda > 0) || !(cov->sigma2 > 0)) return CE_ERR_INVALID_ARG;
    if (cov->kind == CE_COV_MATERN) {
        if (!(cov->nu == 0.5 || cov->nu == 1.5 || cov->nu == 2.5)) return CE_ERR_INVALID_ARG;
    } else if (cov->kind != CE_COV_SEP_EXP) {
        return CE_ERR_INVALID_ARG;
    }
    if (pad->mode < CE_PAD_NONE || pad->mode > CE_PAD_SMOOTH) return CE_ERR_INVALID_ARG;
    const int max_P = pad->max_P > 0 ? std::min(pad->max_P, kMaxP3) : kMaxP3;
    int J = pad->J >= 0 ? pad->J : (pad->mode == CE_PAD_SMOOTH ? n : 0);
    if (pad->mode == CE_PAD_SMOOTH && J < 1) return CE_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);

    double2 *Lc = nullptr;
    double *dstats = nullptr;
    int P = 0;
    double stats[3] = {0, 0, 0};
    auto release = [&]() {
        sce_free(Lc, st);
        sce_free(dstats, st);
        cudaStreamSynchronize(st);
    };
    for (;;) {
        P = 2 * (n + J);
        if (!is_pow2(P) || P < 4 || P > max_P) {
            release();
            return P > max_P ? CE_ERR_NOT_PSD : CE_ERR_INVALID_ARG;
        }
        const long long s = (long long)P * P * P;
        sce_free(Lc, st);
        Lc = nullptr;
        int rc = sce_alloc_t(&Lc, s, st);
        if (rc == CE_OK && !dstats) rc = sce_alloc_t(&dstats, 3, st);
        if (rc != CE_OK) {
            release();
            return rc;
        }
        first_column3_kernel<<<(unsigned)((s + 255) / 256), 256, 0, st>>>(*cov, n, J, P,
                                                                           pad->mode, Lc);
        if ((rc = fft3_f64(Lc, P, st)) != CE_OK) {
            release();
            return rc;
        }
        spectrum3_stats_kernel<<<1, 1024, 0, st>>>(Lc, s, dstats);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(stats, dstats, sizeof(stats), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            release();
            return CE_ERR_CUDA;
        }
        if (stats[0] >= -1e-12 * stats[1]) break;
        if (pad->mode == CE_PAD_NONE || 2 * P > max_P) {
            release();
            return CE_ERR_NOT_PSD;
        }
        J = P - n;   // P -> 2P
    }

    ce3_embedding_s *e = new ce3_embedding_s();
    cudaGetDevice(&e->device);
    e->n = n;
    e->P = P;
    e->J = J;
    e->mode = pad->mode;
    e->cov = *cov;
    e->s = (long long)P * P * P;
    e->lambda_min = stats[0];
    e->lambda_max = stats[1];
    e->max_imag = stats[2];
    e->lam = nullptr;
    e->sq_f = e->sq_c = nullptr;
    const long long s = e->s;
    unsigned char *dmask = nullptr;
    auto fail = [&](int code) {
        sce_free(dmask, st);
        release();
        ce3_destroy(e);
        return code;
    };
    if (cudaMalloc(&e->lam, s * sizeof(double)) != cudaSuccess) return fail(CE_ERR_OOM);
    const unsigned blocks = (unsigned)((s + 255) / 256);
    clip3_kernel<<<blocks, 256, 0, st>>>(Lc, s, e->lam);
    if (cudaGetLastError() != cudaSuccess) return fail(CE_ERR_CUDA);

    // CE_KEEP_TAU_SQRT_S: drop tau = floor(sqrt(s)) eigenvalues (sqrt(s) = P^(3/2))
    auto resolve = [&](long long k) {
        if (k != CE_KEEP_TAU_SQRT_S) return k;
        long long r = (long long)std::sqrt((double)s);
        while (r * r > s) --r;
        while ((r + 1) * (r + 1) <= s) ++r;
        return s - r;
    };
    const long long keep_f = sm ? resolve(sm->keep_fine) : -1;
    const long long keep_c = sm ? resolve(sm->keep_coarse) : -1;
    const double tol = (sm && sm->tie_rel_tol > 0) ? sm->tie_rel_tol : 1e-10;
    const bool need_f = keep_f >= 0 && keep_f < s;
    const bool need_c = keep_c >= 0 && keep_c < s;
    {
        std::vector<double> hl;
        if (need_f || need_c) {
            hl.resize(s);
            if (cudaMemcpyAsync(hl.data(), e->lam, s * sizeof(double), cudaMemcpyDeviceToHost,
                                st) != cudaSuccess ||
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
    }
    if (!need_f) e->mask_f.assign(s, 1);
    if (!need_c) e->mask_c.assign(s, 1);
    e->coarse_distinct = e->mask_c != e->mask_f;

    if (sce_alloc_t(&dmask, s, st) != CE_OK) return fail(CE_ERR_OOM);
    if (cudaMalloc(&e->sq_f, s * sizeof(float)) != cudaSuccess) return fail(CE_ERR_OOM);
    if (cudaMemcpyAsync(dmask, e->mask_f.data(), s, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(CE_ERR_CUDA);
    sqrt3_table_kernel<<<blocks, 256, 0, st>>>(e->lam, dmask, s, e->sq_f);
    if (e->coarse_distinct) {
        if (cudaMalloc(&e->sq_c, s * sizeof(float)) != cudaSuccess) return fail(CE_ERR_OOM);
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CE_ERR_CUDA);
        if (cudaMemcpyAsync(dmask, e->mask_c.data(), s, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return fail(CE_ERR_CUDA);
        sqrt3_table_kernel<<<blocks, 256, 0, st>>>(e->lam, dmask, s, e->sq_c);
    } else {
        e->sq_c = e->sq_f;
    }
    if (cudaGetLastError() != cudaSuccess) return fail(CE_ERR_CUDA);
    sce_free(dmask, st);
    dmask = nullptr;
    release();
    Lc = nullptr;
    dstats = nullptr;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        ce3_destroy(e);
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

extern "C" int ce3_get_eigenvalues(ce3_embedding_t e, double *dst, int dst_on_device,
                                   void *stream) {
    if (!e || !dst) return CE_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    SCE_CUDA(cudaMemcpyAsync(dst, e->lam, e->s * sizeof(double),
                             dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             st));
    if (!dst_on_device) SCE_CUDA(cudaStreamSynchronize(st));
    return CE_OK;
}

extern "C" int ce3_get_mask(ce3_embedding_t e, int which, unsigned char *dst_host) {
    if (!e || !dst_host || which < 0 || which > 1) return CE_ERR_INVALID_ARG;
    const std::vector<unsigned char> &m = which == 0 ? e->mask_f : e->mask_c;
    std::memcpy(dst_host, m.data(), m.size());
    return CE_OK;
}

extern "C" int ce3_get_info(ce3_embedding_t e, ce_embedding_info *info) {
    if (!e || !info) return CE_ERR_INVALID_ARG;
    info->n = e->n;
    info->P = e->P;
    info->J = e->J;
    info->s = e->s;
    info->keep_eff_fine = e->keep_eff_fine;
    info->keep_eff_coarse = e->keep_eff_coarse;
    info->lambda_min = e->lambda_min;
    info->lambda_max = e->lambda_max;
    info->max_imag = e->max_imag;
    return CE_OK;
}

extern "C" int ce3_sample_batch(ce3_embedding_t e, uint64_t seed, uint32_t level,
                                uint64_t first_sample, int count, float *k_fine, float *k_coarse,
                                void *stream) {
    if (!e || count < 0) return CE_ERR_INVALID_ARG;
    if (count == 0 || (!k_fine && !k_coarse)) return CE_OK;
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    if (dev != e->device) return CE_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    int status = CE_OK;
    const float2 *tw = sce_twiddles32(e->P, &status);
    if (status != CE_OK) return status;
    const int P = e->P, m = e->n, mc = m / 2;
    const bool masked = e->coarse_distinct && k_coarse != nullptr;
    const bool need_fine = k_fine != nullptr || (!masked && k_coarse != nullptr);
    const size_t y1 = (size_t)(m + 1) * P * P, y2 = (size_t)(m + 1) * (m + 1) * P;
    const size_t y1c = masked ? (size_t)(mc + 1) * P * P : 0;
    const size_t y2c = masked ? (size_t)(mc + 1) * (mc + 1) * P : 0;
    const size_t kv = (size_t)(m + 1) * (m + 1) * (m + 1);
    const size_t per_sample = (y1 + y2 + y1c + y2c) * sizeof(float2) +
                              (k_fine ? 0 : kv * sizeof(float));
    int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)count, (1ull << 30) / per_sample));
    chunk = std::min(chunk, 65535);
    float2 *Y1 = nullptr, *Y2 = nullptr, *Y1c = nullptr, *Y2c = nullptr;
    float *kf_tmp = nullptr;
    int rc = sce_alloc_t(&Y1, chunk * y1, st);
    if (rc == CE_OK) rc = sce_alloc_t(&Y2, chunk * y2, st);
    if (rc == CE_OK && masked) rc = sce_alloc_t(&Y1c, chunk * y1c, st);
    if (rc == CE_OK && masked) rc = sce_alloc_t(&Y2c, chunk * y2c, st);
    if (rc == CE_OK && need_fine && !k_fine) rc = sce_alloc_t(&kf_tmp, chunk * kv, st);
    const Cfg3 cx = cfg3(P, masked ? (long long)P * P : (long long)P * P / 2);
    for (int c0 = 0; c0 < count && rc == CE_OK; c0 += chunk) {
        const int cn = std::min(chunk, count - c0);
        float *kf_c = k_fine ? k_fine + (size_t)c0 * kv : kf_tmp;
        float *kc_c = k_coarse ? k_coarse + (size_t)c0 * (mc + 1) * (mc + 1) * (mc + 1) : nullptr;
        rc = cx.maxb == 4
                 ? launch_x3<4>(e, masked, tw, seed, level, first_sample + c0, cn, Y1, Y1c, cx, st)
                 : launch_x3<8>(e, masked, tw, seed, level, first_sample + c0, cn, Y1, Y1c, cx, st);
        if (rc != CE_OK) break;
        if (need_fine) {
            rc = launch_y3(Y1, m + 1, P, m + 1, 1, tw, cn, Y2, st);
            if (rc == CE_OK)
                rc = launch_z3(Y2, m + 1, m + 1, P, m + 1, 1, tw, cn, kf_c,
                               masked ? nullptr : kc_c, mc, st);
        }
        if (rc == CE_OK && masked) {
            rc = launch_y3(Y1c, mc + 1, P, mc + 1, 2, tw, cn, Y2c, st);
            if (rc == CE_OK)
                rc = launch_z3(Y2c, mc + 1, mc + 1, P, mc + 1, 2, tw, cn, kc_c, nullptr, mc, st);
        }
    }
    sce_free(Y1, st);
    sce_free(Y2, st);
    sce_free(Y1c, st);
    sce_free(Y2c, st);
    sce_free(kf_tmp, st);
    return rc;
}

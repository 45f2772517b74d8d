// Darcy problem on the unit cube (§3.1-3.2 in d = 3) and the MLMC level
// estimate built on it.
//
//   -div(k grad u) = f on (0,1)^3, u = 1 at x1 = 0, u = 0 at x1 = 1, zero
//   flux on the other faces; P1 elements on the six Kuhn tetrahedra of every
//   cell, k averaged over each tetrahedron's four vertices.
//
// Operator.  For the Kuhn tetrahedron {a, a+e_p0, a+e_p0+e_p1, a+(1,1,1)} the
// barycentric gradients are -e_p0/h, (e_p0-e_p1)/h, (e_p1-e_p2)/h, e_p2/h, so
// only the three path edges (all axis-parallel) have a non-zero stiffness
// entry, -|T|/h^2 = -h/6.  The stiffness matrix is therefore a seven-point
// stencil whose edge conductance is (h/6) sum over the tetrahedra containing
// the edge of kbar_T = (h/24) sum_T sum_{v in T} k_v.  An edge along axis e
// from vertex p lies in (a1, a2 the other two axes; a term only where its cell
// exists):
//   cell p          : {p, p+e, p+e+a1, p+e+a1+a2}, {p, p+e, p+e+a2, p+e+a1+a2}
//   cell p-a1       : {p-a1, p, p+e, p+e+a2}
//   cell p-a2       : {p-a2, p, p+e, p+e+a1}
//   cell p-a1-a2    : {p-a1-a2, p-a2, p, p+e}, {p-a1-a2, p-a1, p, p+e}
// The system is divided by h: conductances g = S/24 (S the vertex sum above)
// and load F'_p = f h^2 N(p)/24, N(p) = number of tetrahedra at p (6 for the
// cell corners a and a+(1,1,1) of each adjacent cell, 2 for the others).
//
// Solver: iterative refinement; the residual F' - A'u is formed in
// float-float (pairs of FP32 numbers, ~48 significant bits) from float-float
// conductances and u, the correction solves A'd = r by FP32 CG
// preconditioned with one geometric multigrid V(1,1) cycle (red-black
// Gauss-Seidel in the (i+j+k) parity, full-weighting restriction, trilinear
// prolongation, coarse conductances from two fine edges in series averaged
// over the 3x3 transverse lines with weights 1, 1/2; exact solve of the 9
// unknowns of the 2-cell grid).  Per-sample flags stop converged samples, so a
// sample's result does not depend on the batch it is solved in.
//
// The multigrid cycle reads FP16 copies of its conductances (the smoother,
// residual and transfers are streaming passes); it is then a fixed symmetric
// preconditioner for a nearby operator, while CG applies the FP32 operator and
// the refinement the FP64 one, so the converged solution is unchanged.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ff.cuh"
#include "sce_internal.cuh"

using sce::ff;
using sce::ff_add;
using sce::ff_add_f;
using sce::ff_from_double;
using sce::ff_mul;
using sce::ff_sub;
using sce::two_prod;

namespace {

constexpr int MAXLEV3 = 9;    // n <= 256
constexpr int TPB3 = 256;
constexpr int VPT3 = 8;
constexpr int EPB3 = TPB3 * VPT3;

// vertex index within one sample -> (i, j, k); 32-bit arithmetic (a sample
// has at most 257^3 vertices)
__device__ __forceinline__ void decode3(int v, int w, int *i, int *j, int *k) {
    const unsigned r = (unsigned)v / (unsigned)w;
    *i = v - (int)r * w;
    *k = (int)(r / (unsigned)w);
    *j = (int)r - *k * w;
}

template <int E> struct Axes {
    static constexpr int A1 = (E + 1) % 3, A2 = (E + 2) % 3;
};

__device__ __forceinline__ long long stride3(int axis, int w) {
    return axis == 0 ? 1 : (axis == 1 ? (long long)w : (long long)w * w);
}

// S of the edge along axis E from (c0, c1, c2) (see the file comment); 0 on
// the last plane of E.  The at most 24 FP32 terms are summed in float-float
// (each term added with an error-free two-sum), so the FP64 value hi + lo is
// the sum to ~2^-48 relative without FP64 additions (FP64 runs at a small
// fraction of the FP32 rate on this GPU).
template <int E>
__device__ __forceinline__ double edge_sum3(const float *__restrict__ ks, int n, const int c[3],
                                            long long v) {
    constexpr int A1 = Axes<E>::A1, A2 = Axes<E>::A2;
    if (c[E] >= n) return 0.0;
    const int w = n + 1;
    const long long se = stride3(E, w), s1 = stride3(A1, w), s2 = stride3(A2, w);
    auto K = [&](int de, int d1, int d2) { return ks[v + de * se + d1 * s1 + d2 * s2]; };
    const bool lo1 = c[A1] > 0, hi1 = c[A1] < n, lo2 = c[A2] > 0, hi2 = c[A2] < n;
    const float k0 = K(0, 0, 0), ke = K(1, 0, 0);
    int cnt = 0;   // multiplicity of k0 and ke: one per tetrahedron
    ff S = {0.0f, 0.0f};
    if (hi1 && hi2) {
        cnt += 2;
        S = ff_add_f(S, K(1, 1, 0));
        S = ff_add_f(S, K(1, 0, 1));
        S = ff_add_f(S, 2.0f * K(1, 1, 1));
    }
    if (lo1 && hi2) {
        cnt += 1;
        S = ff_add_f(S, K(0, -1, 0));
        S = ff_add_f(S, K(1, 0, 1));
    }
    if (hi1 && lo2) {
        cnt += 1;
        S = ff_add_f(S, K(0, 0, -1));
        S = ff_add_f(S, K(1, 1, 0));
    }
    if (lo1 && lo2) {
        cnt += 2;
        S = ff_add_f(S, 2.0f * K(0, -1, -1));
        S = ff_add_f(S, K(0, 0, -1));
        S = ff_add_f(S, K(0, -1, 0));
    }
    // cnt (k0 + ke): cnt <= 6, each product cnt * k exact in FP32 up to a
    // 3-bit growth of the significand, added as two terms
    S = ff_add(S, two_prod((float)cnt, k0));
    S = ff_add(S, two_prod((float)cnt, ke));
    return (double)S.hi + (double)S.lo;
}

// tetrahedra at vertex (i, j, k) of an n-cell grid
__device__ __forceinline__ int tets_at(int i, int j, int k, int n) {
    int N = 0;
    for (int d = 0; d < 8; ++d) {
        const int di = d & 1, dj = (d >> 1) & 1, dk = (d >> 2) & 1;
        const bool ok = (di ? i > 0 : i < n) && (dj ? j > 0 : j < n) && (dk ? k > 0 : k < n);
        if (ok) N += (d == 0 || d == 7) ? 6 : 2;
    }
    return N;
}

// ---------------------------------------------------------------- per-vertex kernels
// grid: (blocks over vertices, samples); a thread visits VPT3 vertices
#define FOR_V3(V)                                                                          \
    _Pragma("unroll") for (int e_ = 0; e_ < VPT3; ++e_)                                    \
        if (const int v = (int)blockIdx.x * EPB3 + (int)threadIdx.x + e_ * TPB3; v < (int)(V))

// conductances g = S/24 as float-float: hi (the FP32 operator of CG) and lo
__global__ void cond3_kernel(const float *__restrict__ k, int n, float *__restrict__ gx,
                             float *__restrict__ gy, float *__restrict__ gz,
                             float *__restrict__ glx, float *__restrict__ gly,
                             float *__restrict__ glz) {
    const int s = blockIdx.y;
    const int w = n + 1;
    const long long V = (long long)w * w * w, off = (long long)s * V;
    const float *ks = k + off;
    FOR_V3(V) {
        int c[3];
        decode3(v, w, &c[0], &c[1], &c[2]);
        const double x = edge_sum3<0>(ks, n, c, v) * (1.0 / 24.0);
        const double y = edge_sum3<1>(ks, n, c, v) * (1.0 / 24.0);
        const double z = edge_sum3<2>(ks, n, c, v) * (1.0 / 24.0);
        const ff fx = ff_from_double(x), fy = ff_from_double(y), fz = ff_from_double(z);
        gx[off + v] = fx.hi;
        gy[off + v] = fy.hi;
        gz[off + v] = fz.hi;
        glx[off + v] = fx.lo;
        gly[off + v] = fy.lo;
        glz[off + v] = fz.lo;
    }
}

__device__ __forceinline__ float series3(float a, float b) {
    const float t = a + b;
    return t > 0.0f ? a * b / t : 0.0f;
}

// coarse conductance along axis E at coarse vertex c (coarse grid nc = nf/2):
// two fine edges in series, averaged over the transverse fine lines with
// weights 1 (through the coarse line) and 1/2 (its neighbours)
template <int E>
__device__ __forceinline__ float coarse_cond3(const float *__restrict__ gf, int nf, const int c[3]) {
    constexpr int A1 = Axes<E>::A1, A2 = Axes<E>::A2;
    const int nc = nf / 2;
    if (c[E] >= nc) return 0.0f;
    const int wf = nf + 1;
    const long long se = stride3(E, wf), s1 = stride3(A1, wf), s2 = stride3(A2, wf);
    const long long base = 2 * (c[0] * stride3(0, wf) + c[1] * stride3(1, wf) + c[2] * stride3(2, wf));
    float acc = 0.0f;
    for (int d2 = -1; d2 <= 1; ++d2) {
        const int f2 = 2 * c[A2] + d2;
        if (f2 < 0 || f2 > nf) continue;
        const float w2 = d2 == 0 ? 1.0f : 0.5f;
        for (int d1 = -1; d1 <= 1; ++d1) {
            const int f1 = 2 * c[A1] + d1;
            if (f1 < 0 || f1 > nf) continue;
            const float w1 = d1 == 0 ? 1.0f : 0.5f;
            const long long q = base + d1 * s1 + d2 * s2;
            acc += w1 * w2 * series3(gf[q], gf[q + se]);
        }
    }
    return acc;
}

__global__ void coarsen3_kernel(const float *__restrict__ fx, const float *__restrict__ fy,
                                const float *__restrict__ fz, int nf, float *__restrict__ cx,
                                float *__restrict__ cy, float *__restrict__ cz,
                                __half *__restrict__ hx, __half *__restrict__ hy,
                                __half *__restrict__ hz) {
    const int s = blockIdx.y;
    const int nc = nf / 2, wc = nc + 1, wf = nf + 1;
    const long long Vc = (long long)wc * wc * wc, Vf = (long long)wf * wf * wf;
    const float *ax = fx + s * Vf, *ay = fy + s * Vf, *az = fz + s * Vf;
    FOR_V3(Vc) {
        int c[3];
        decode3(v, wc, &c[0], &c[1], &c[2]);
        const float x = coarse_cond3<0>(ax, nf, c), y = coarse_cond3<1>(ay, nf, c),
                    z = coarse_cond3<2>(az, nf, c);
        cx[s * Vc + v] = x;
        cy[s * Vc + v] = y;
        cz[s * Vc + v] = z;
        hx[s * Vc + v] = __float2half_rn(x);
        hy[s * Vc + v] = __float2half_rn(y);
        hz[s * Vc + v] = __float2half_rn(z);
    }
}

__device__ __forceinline__ float gval(float x) { return x; }
__device__ __forceinline__ float gval(__half x) { return __half2float(x); }

// sum of g_e (z_p - z_q) over the six edges of an unknown vertex
template <typename T, typename Tg>
__device__ __forceinline__ T apply3(const Tg *gx, const Tg *gy, const Tg *gz, const T *z,
                                    long long v, int j, int k, int n) {
    const int w = n + 1;
    const long long w2 = (long long)w * w;
    const T zc = z[v];
    T a = (T)gval(gx[v - 1]) * (zc - z[v - 1]) + (T)gval(gx[v]) * (zc - z[v + 1]);
    if (j > 0) a += (T)gval(gy[v - w]) * (zc - z[v - w]);
    if (j < n) a += (T)gval(gy[v]) * (zc - z[v + w]);
    if (k > 0) a += (T)gval(gz[v - w2]) * (zc - z[v - w2]);
    if (k < n) a += (T)gval(gz[v]) * (zc - z[v + w2]);
    return a;
}

__global__ void half3_kernel(const float *__restrict__ gx, const float *__restrict__ gy,
                             const float *__restrict__ gz, long long total,
                             __half *__restrict__ hx, __half *__restrict__ hy,
                             __half *__restrict__ hz) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        hx[i] = __float2half_rn(gx[i]);
        hy[i] = __float2half_rn(gy[i]);
        hz[i] = __float2half_rn(gz[i]);
    }
}

// Row-structured launches of the stencil kernels: a row is the grid line
// (j, k); 2^lt threads per row (at least its work items), 256 / 2^lt rows per
// block, grid (rows, samples).  One division per thread, 32-bit offsets from
// the sample's base pointers.
__device__ __forceinline__ bool row3(int w, int lt, int *t, int *j, int *k) {
    const int row = blockIdx.x * (256 >> lt) + (threadIdx.x >> lt);
    if (row >= w * w) return false;
    *t = threadIdx.x & ((1 << lt) - 1);
    *k = (int)((unsigned)row / (unsigned)w);
    *j = row - *k * w;
    return true;
}

// red-black Gauss-Seidel half-sweep of colour `color` ((i + j + k) % 2): n/2
// threads per row, i = 2t + parity.  FROM_ZERO: the first half-sweep from
// z = 0 (z = b/diag at the colour's unknowns and 0 at the other colour's,
// so z is not read and needs no clearing).  The Dirichlet planes i = 0, n
// are never written: z there is zeroed once when the hierarchy is allocated.
// The division is the fast single-precision one: the smoother only has to be
// a fixed symmetric operation, not correctly rounded.
template <typename Tg, bool FROM_ZERO>
__global__ void __launch_bounds__(256) smooth3_kernel(
    const Tg *__restrict__ gx, const Tg *__restrict__ gy, const Tg *__restrict__ gz,
    const float *__restrict__ b, float *__restrict__ z, int n, int lt, int color,
    const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int w = n + 1, w2 = w * w;
    int t, j, k;
    if (!row3(w, lt, &t, &j, &k)) return;
    const long long off = (long long)s * w2 * w;
    const Tg *ax = gx + off, *ay = gy + off, *az = gz + off;
    const float *bs = b + off;
    float *zs = z + off;
    const int par = (color + j + k) & 1;
    const int rowv = (k * w + j) * w;
    if (FROM_ZERO) {
        const int io = 2 * t + (1 - par);
        if (io >= 1) zs[rowv + io] = 0.0f;
    }
    const int i = 2 * t + par;
    if (i < 1) return;
    const int v = rowv + i;
    const float cw = gval(ax[v - 1]), ce = gval(ax[v]);
    const float cs = j > 0 ? gval(ay[v - w]) : 0.0f, cn = j < n ? gval(ay[v]) : 0.0f;
    const float cd = k > 0 ? gval(az[v - w2]) : 0.0f, cu = k < n ? gval(az[v]) : 0.0f;
    const float d = cw + ce + cs + cn + cd + cu;
    if (FROM_ZERO) {
        zs[v] = __fdividef(bs[v], d);
    } else {
        float acc = bs[v] + cw * zs[v - 1] + ce * zs[v + 1];
        if (j > 0) acc += cs * zs[v - w];
        if (j < n) acc += cn * zs[v + w];
        if (k > 0) acc += cd * zs[v - w2];
        if (k < n) acc += cu * zs[v + w2];
        zs[v] = __fdividef(acc, d);
    }
}

// res = b - A z at the unknowns (n threads per row, i = 1 + t); the
// Dirichlet planes of res are never read
template <typename Tg>
__global__ void __launch_bounds__(256) resid3_kernel(
    const Tg *__restrict__ gx, const Tg *__restrict__ gy, const Tg *__restrict__ gz,
    const float *__restrict__ b, const float *__restrict__ z, float *__restrict__ res, int n,
    int lt, const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int w = n + 1;
    int t, j, k;
    if (!row3(w, lt, &t, &j, &k) || t >= n - 1) return;
    const long long off = (long long)s * w * w * w;
    const int v = (k * w + j) * w + 1 + t;
    res[off + v] = b[off + v] - apply3(gx + off, gy + off, gz + off, z + off, (long long)v, j, k, n);
}

// coarse right-hand side by full weighting (the transpose of trilinear
// prolongation) at coarse unknowns (nc threads per coarse row, I = 1 + t);
// the coarse Dirichlet planes of bc are never read
__global__ void __launch_bounds__(256) restrict3_kernel(const float *__restrict__ res, int nf,
                                                        float *__restrict__ bc, int lt,
                                                        const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int nc = nf / 2, wc = nc + 1, wf = nf + 1;
    int t, J, K;
    if (!row3(wc, lt, &t, &J, &K) || t >= nc - 1) return;
    const int I = 1 + t;
    const float *rs = res + (long long)s * wf * wf * wf;
    float acc = 0.0f;
    for (int dk = -1; dk <= 1; ++dk) {
        const int k = 2 * K + dk;
        if (k < 0 || k > nf) continue;
        const float wk = dk == 0 ? 1.0f : 0.5f;
        for (int dj = -1; dj <= 1; ++dj) {
            const int j = 2 * J + dj;
            if (j < 0 || j > nf) continue;
            const float wj = dj == 0 ? 1.0f : 0.5f;
            const int row = (k * wf + j) * wf + 2 * I;
            acc += wk * wj * (0.5f * rs[row - 1] + rs[row] + 0.5f * rs[row + 1]);
        }
    }
    bc[(long long)s * wc * wc * wc + (K * wc + J) * wc + I] = acc;
}

// z += trilinear interpolation of the coarse correction (unknowns only; nf
// threads per fine row, i = 1 + t)
__global__ void __launch_bounds__(256) prolong3_kernel(const float *__restrict__ zc, int nc,
                                                       float *__restrict__ zf, int lt,
                                                       const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int nf = 2 * nc, wf = nf + 1, wc = nc + 1;
    int t, j, k;
    if (!row3(wf, lt, &t, &j, &k) || t >= nf - 1) return;
    const int i = 1 + t;
    const float *c = zc + (long long)s * wc * wc * wc;
    // the coarse neighbours (a >> 1, (a + 1) >> 1) per axis coincide on
    // even fine indices, so the eight-term mean is the trilinear weight
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const int i1 = (i + 1) >> 1, j1 = (j + 1) >> 1, k1 = (k + 1) >> 1;
    const float *c00 = c + (k0 * wc + j0) * wc, *c01 = c + (k0 * wc + j1) * wc;
    const float *c10 = c + (k1 * wc + j0) * wc, *c11 = c + (k1 * wc + j1) * wc;
    const float acc = ((c00[i0] + c00[i1]) + (c01[i0] + c01[i1])) +
                      ((c10[i0] + c10[i1]) + (c11[i0] + c11[i1]));
    zf[(long long)s * wf * wf * wf + (k * wf + j) * wf + i] += 0.125f * acc;
}

// exact solve on the 2-cell grid: unknowns (1, j, k), j, k = 0..2, one
// thread per sample, Gaussian elimination of the 9 x 9 SPD system
__global__ void coarsest3_kernel(const float *__restrict__ gx, const float *__restrict__ gy,
                                 const float *__restrict__ gz, const float *__restrict__ b,
                                 float *__restrict__ z, int count, const int *__restrict__ act) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count || !act[s]) return;
    const long long off = (long long)s * 27;
    float A[9][9], r[9];
    for (int a = 0; a < 9; ++a) {
        for (int c = 0; c < 9; ++c) A[a][c] = 0.0f;
    }
    for (int k = 0; k < 3; ++k) {
        for (int j = 0; j < 3; ++j) {
            const int u = j + 3 * k;
            const long long v = off + (k * 3 + j) * 3 + 1;
            float d = gx[v - 1] + gx[v];
            if (j > 0) d += gy[v - 3];
            if (j < 2) {
                d += gy[v];
                A[u][u + 1] = A[u + 1][u] = -gy[v];
            }
            if (k > 0) d += gz[v - 9];
            if (k < 2) {
                d += gz[v];
                A[u][u + 3] = A[u + 3][u] = -gz[v];
            }
            A[u][u] = d;
            r[u] = b[v];
        }
    }
    for (int p = 0; p < 9; ++p) {
        for (int q = p + 1; q < 9; ++q) {
            const float m = A[q][p] / A[p][p];
            for (int c = p; c < 9; ++c) A[q][c] -= m * A[p][c];
            r[q] -= m * r[p];
        }
    }
    float x[9];
    for (int p = 8; p >= 0; --p) {
        float t = r[p];
        for (int c = p + 1; c < 9; ++c) t -= A[p][c] * x[c];
        x[p] = t / A[p][p];
    }
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) z[off + (k * 3 + j) * 3 + 1] = x[j + 3 * k];
}

// ---------------------------------------------------------------- Krylov pieces
__device__ __forceinline__ float block_sum3(float v, float *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;
}

// q = A p at the unknowns (q on the Dirichlet planes stays 0 from the clear at
// allocation), partial p.q per block
__global__ void __launch_bounds__(TPB3) spmv_dot3_kernel(
    const float *__restrict__ gx, const float *__restrict__ gy, const float *__restrict__ gz,
    const float *__restrict__ p, float *__restrict__ q, int n, double *__restrict__ part,
    int nblk, const int *__restrict__ act) {
    __shared__ float sh[32];
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int w = n + 1;
    const long long V = (long long)w * w * w, off = (long long)s * V;
    float acc = 0.0f;
    FOR_V3(V) {
        int i, j, k;
        decode3(v, w, &i, &j, &k);
        if (i > 0 && i < n) {
            const float val = apply3(gx + off, gy + off, gz + off, p + off, (long long)v, j, k, n);
            acc += p[off + v] * val;
            q[off + v] = val;
        }
    }
    const float tot = block_sum3(acc, sh);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = (double)tot;
}

__global__ void __launch_bounds__(TPB3) axpy2_3_kernel(
    float *__restrict__ d, float *__restrict__ r, const float *__restrict__ p,
    const float *__restrict__ q, const double *__restrict__ alpha, long long V,
    double *__restrict__ part, int nblk, const int *__restrict__ act) {
    __shared__ float sh[32];
    const int s = blockIdx.y;
    if (!act[s]) return;
    const float a = (float)alpha[s];
    const long long off = (long long)s * V;
    float acc = 0.0f;
    FOR_V3(V) {
        const long long g = off + v;
        d[g] += a * p[g];
        const float rv = r[g] - a * q[g];
        r[g] = rv;
        acc += rv * rv;
    }
    const float tot = block_sum3(acc, sh);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = (double)tot;
}

__global__ void __launch_bounds__(TPB3) dot3_kernel(const float *__restrict__ a,
                                                    const float *__restrict__ b, long long V,
                                                    double *__restrict__ part, int nblk,
                                                    const int *__restrict__ act) {
    __shared__ float sh[32];
    const int s = blockIdx.y;
    if (!act[s]) return;
    const long long off = (long long)s * V;
    float acc = 0.0f;
    FOR_V3(V) acc += a[off + v] * b[off + v];
    const float tot = block_sum3(acc, sh);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = (double)tot;
}

// p = z + beta p (first == 1: p = z)
__global__ void __launch_bounds__(TPB3) pupdate3_kernel(float *__restrict__ p,
                                                        const float *__restrict__ z,
                                                        const double *__restrict__ beta,
                                                        long long V, int first,
                                                        const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const float bt = first ? 0.0f : (float)beta[s];
    const long long off = (long long)s * V;
    FOR_V3(V) {
        const long long g = off + v;
        p[g] = first ? z[g] : z[g] + bt * p[g];
    }
}

// ---------------------------------------------------------------- reductions
struct Scal3 {
    double *rz, *pq, *rr, *alpha, *beta, *orr, *orr0, *thr;
    int *act_out, *act_in, *iters, *counter;
};

enum { R3_ALPHA = 0, R3_RR = 1, R3_BETA = 2, R3_RZ0 = 3, R3_ORR = 4, R3_ORR0 = 5 };

// one warp per sample: fixed-order sum of the block partials, then the
// scalar update of `mode`
__global__ void reduce3_kernel(const double *__restrict__ part, int nblk, int count, int mode,
                               Scal3 sc, const int *__restrict__ act, double rtol2,
                               double in_rel2) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= count) return;
    const int s = warp;
    if (act && !act[s]) return;
    double v = 0.0;
    for (int i = lane; i < nblk; i += 32) v += part[(long long)s * nblk + i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane != 0) return;
    switch (mode) {
        case R3_ALPHA:
            sc.pq[s] = v;
            sc.alpha[s] = v > 0.0 ? sc.rz[s] / v : 0.0;
            break;
        case R3_RR: {
            sc.rr[s] = v;
            sc.iters[s] += 1;
            if (!(v > sc.thr[s])) sc.act_in[s] = 0;
            else atomicAdd(sc.counter, 1);
            break;
        }
        case R3_BETA:
            sc.beta[s] = sc.rz[s] > 0.0 ? v / sc.rz[s] : 0.0;
            sc.rz[s] = v;
            break;
        case R3_RZ0:
            sc.rz[s] = v;
            break;
        default: {   // R3_ORR, R3_ORR0
            sc.orr[s] = v;
            if (mode == R3_ORR0) sc.orr0[s] = v;
            const bool more = v > rtol2 * sc.orr0[s] && v == v;
            sc.act_out[s] = more ? 1 : 0;
            sc.act_in[s] = sc.act_out[s];
            sc.thr[s] = fmax(in_rel2 * v, 0.0625 * rtol2 * sc.orr0[s]);
            if (more) atomicAdd(sc.counter, 1);
            break;
        }
    }
}

// ---------------------------------------------------------------- refinement (float-float)
// u and the conductances as float-float (hi, lo): ~48 significant bits, with
// FP32 instructions only (FP64 runs at a small fraction of the FP32 rate)
struct Outer3 {
    const float *gx, *gy, *gz, *glx, *gly, *glz;
    float2 *u;
};

__global__ void lift3_kernel(float2 *__restrict__ u, int n) {
    const int s = blockIdx.y;
    const int w = n + 1;
    const long long V = (long long)w * w * w, off = (long long)s * V;
    FOR_V3(V) u[off + v] = make_float2((v % w == 0) ? 1.0f : 0.0f, 0.0f);
}

// (A'u)_p of an unknown vertex in float-float (differences of u formed first)
__device__ __forceinline__ ff apply3_ff(const Outer3 &o, long long v, int j, int k, int n) {
    const int w = n + 1;
    const long long w2 = (long long)w * w;
    auto U = [&](long long q) {
        const float2 t = o.u[q];
        return ff{t.x, t.y};
    };
    const ff uc = U(v);
    ff a = ff_mul(ff{o.gx[v - 1], o.glx[v - 1]}, ff_sub(uc, U(v - 1)));
    a = ff_add(a, ff_mul(ff{o.gx[v], o.glx[v]}, ff_sub(uc, U(v + 1))));
    if (j > 0) a = ff_add(a, ff_mul(ff{o.gy[v - w], o.gly[v - w]}, ff_sub(uc, U(v - w))));
    if (j < n) a = ff_add(a, ff_mul(ff{o.gy[v], o.gly[v]}, ff_sub(uc, U(v + w))));
    if (k > 0) a = ff_add(a, ff_mul(ff{o.gz[v - w2], o.glz[v - w2]}, ff_sub(uc, U(v - w2))));
    if (k < n) a = ff_add(a, ff_mul(ff{o.gz[v], o.glz[v]}, ff_sub(uc, U(v + w2))));
    return a;
}

// r = F' - A'u at unknowns -> b (FP32), partial |r|^2 (FP64); samples with act == 0 skip
__global__ void __launch_bounds__(TPB3) outer_residual3_kernel(
    Outer3 o, int n, double fh2, float *__restrict__ b, double *__restrict__ part, int nblk,
    const int *__restrict__ act) {
    __shared__ double shd[32];
    const int s = blockIdx.y;
    if (act && !act[s]) return;
    const int w = n + 1;
    const long long V = (long long)w * w * w, off = (long long)s * V;
    Outer3 os = o;
    os.gx += off;
    os.gy += off;
    os.gz += off;
    os.glx += off;
    os.gly += off;
    os.glz += off;
    os.u += off;
    double acc = 0.0;
    FOR_V3(V) {
        int i, j, k;
        decode3(v, w, &i, &j, &k);
        float rb = 0.0f;
        if (i > 0 && i < n) {
            const ff r = ff_sub(ff_from_double(fh2 * (double)tets_at(i, j, k, n) * (1.0 / 24.0)),
                                apply3_ff(os, v, j, k, n));
            rb = r.hi + r.lo;
            const double rd = (double)r.hi + (double)r.lo;
            acc += rd * rd;
        }
        b[off + v] = rb;
    }
    for (int q = 16; q > 0; q >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, q);
    if ((threadIdx.x & 31) == 0) shd[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += shd[i];
        part[(long long)s * nblk + blockIdx.x] = t;
    }
}

__global__ void outer_update3_kernel(float2 *__restrict__ u, const float *__restrict__ d, int n,
                                     const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int w = n + 1;
    const long long V = (long long)w * w * w, off = (long long)s * V;
    FOR_V3(V) {
        const int i = v % w;
        if (i > 0 && i < n) {
            const float2 t = u[off + v];
            const ff r = ff_add_f(ff{t.x, t.y}, d[off + v]);
            u[off + v] = make_float2(r.hi, r.lo);
        }
    }
}

// u = u0 (FP64 nodal values, Dirichlet planes included) as float-float
__global__ void set_u3_kernel(float2 *__restrict__ u, const double *__restrict__ u0,
                              long long total) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const ff t = ff_from_double(u0[q]);
        u[q] = make_float2(t.hi, t.lo);
    }
}

// trilinear prolongation of the coarse solution (nc cells per side) to the
// fine grid: the first iterate of the fine solve of the same field
__global__ void prolong_u3_kernel(const double *__restrict__ uc, int nc, int count,
                                  double *__restrict__ uf) {
    const int nf = 2 * nc, wf = nf + 1, wc = nc + 1;
    const long long Vf = (long long)wf * wf * wf, Vc = (long long)wc * wc * wc;
    const long long total = (long long)count * Vf;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long s = q / Vf;
        int i, j, k;
        decode3((int)(q - s * Vf), wf, &i, &j, &k);
        const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
        const int k0 = k >> 1, k1 = (k + 1) >> 1;
        const double *c = uc + s * Vc;
        auto C = [&](int a, int b, int d) { return c[((long long)d * wc + b) * wc + a]; };
        uf[q] = 0.125 * (((C(i0, j0, k0) + C(i1, j0, k0)) + (C(i0, j1, k0) + C(i1, j1, k0))) +
                         ((C(i0, j0, k1) + C(i1, j0, k1)) + (C(i0, j1, k1) + C(i1, j1, k1))));
    }
}

__global__ void u_to_double3_kernel(const float2 *__restrict__ u, long long total,
                                    double *__restrict__ out) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const float2 t = u[q];
        out[q] = (double)t.x + (double)t.y;
    }
}

// ---------------------------------------------------------------- QoIs (FP64)
// partials of the outflow h sum_{j,k} [g_x(n-1, j, k) u(n-1, j, k) + F'(n, j, k)]
// (over the vertices of the x1 = 1 plane) and of sum_T (sum u_i^2 + (sum u_i)^2)
// over the six tetrahedra of every cell
__global__ void __launch_bounds__(TPB3) qoi3_partial_kernel(
    const float *__restrict__ gx, const float *__restrict__ glx, const double *__restrict__ u,
    int n, double fh2, double *__restrict__ part_out, double *__restrict__ part_l2, int nblk) {
    __shared__ double sa[32], sb[32];
    const int s = blockIdx.y;
    const int w = n + 1;
    const long long V = (long long)w * w * w, off = (long long)s * V;
    const double *us = u + off;
    const long long w2 = (long long)w * w;
    double a = 0.0, b = 0.0;
    FOR_V3(V) {
        int i, j, k;
        decode3(v, w, &i, &j, &k);
        if (i == n)
            a += ((double)gx[off + v - 1] + (double)glx[off + v - 1]) * us[v - 1] +
                 fh2 * (double)tets_at(i, j, k, n) * (1.0 / 24.0);
        if (i < n && j < n && k < n) {
            // corners: bit 0 = +x, bit 1 = +y, bit 2 = +z
            double c[8];
            for (int d = 0; d < 8; ++d) c[d] = us[v + (d & 1) + ((d >> 1) & 1) * w + (d >> 2) * w2];
            // Kuhn tetrahedra 0, e_p0, e_p0 + e_p1, (1,1,1) for the six orders
            const int path[6][2] = {{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 6}};
            for (int t = 0; t < 6; ++t) {
                const double x0 = c[0], x1 = c[path[t][0]], x2 = c[path[t][1]], x3 = c[7];
                const double sum = x0 + x1 + x2 + x3;
                b += x0 * x0 + x1 * x1 + x2 * x2 + x3 * x3 + sum * sum;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        part_out[(long long)s * nblk + blockIdx.x] = ta;
        part_l2[(long long)s * nblk + blockIdx.x] = tb;
    }
}

// QoIs of qmask (bit 0 outflow, 1 point value, 2 L2 norm; the others are
// written as 0; part_out / part_l2 may be NULL when qmask has neither)
__global__ void qoi3_final_kernel(const double *__restrict__ part_out,
                                  const double *__restrict__ part_l2, int nblk, int count,
                                  const double *__restrict__ u, int n, Scal3 sc, double rtol2,
                                  double *__restrict__ qoi, int *__restrict__ iters_out,
                                  int *__restrict__ status_out, int *__restrict__ misc,
                                  int qmask) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= count) return;
    const int s = warp;
    double a = 0.0, b = 0.0;
    for (int i = lane; part_out && i < nblk; i += 32) {
        a += part_out[(long long)s * nblk + i];
        b += part_l2[(long long)s * nblk + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane != 0) return;
    const double h = 1.0 / (double)n;
    const int w = n + 1;
    const long long off = (long long)s * w * w * w;
    // point value at (7/15)^3: cell a, local t; the Kuhn tetrahedron of the
    // descending order of the local coordinates
    const double xs = 7.0 / 15.0 * (double)n;
    const int ca = min((int)floor(xs), n - 1);
    double t[3] = {xs - ca, xs - ca, xs - ca};
    int ord[3] = {0, 1, 2};
    for (int p = 0; p < 3; ++p)
        for (int q = p + 1; q < 3; ++q)
            if (t[ord[q]] > t[ord[p]]) {
                const int tmp = ord[p];
                ord[p] = ord[q];
                ord[q] = tmp;
            }
    int c[3] = {ca, ca, ca};
    auto U = [&](const int *cc) { return u[off + ((long long)cc[2] * w + cc[1]) * w + cc[0]]; };
    double q_pt = (1.0 - t[ord[0]]) * U(c);
    c[ord[0]] += 1;
    q_pt += (t[ord[0]] - t[ord[1]]) * U(c);
    c[ord[1]] += 1;
    q_pt += (t[ord[1]] - t[ord[2]]) * U(c);
    c[ord[2]] += 1;
    q_pt += t[ord[2]] * U(c);
    const double q_out = h * a;
    const double q_l2 = sqrt(b * h * h * h / 120.0);   // |T| / 20 = h^3 / 120
    qoi[3 * s + 0] = (qmask & 1) ? q_out : 0.0;
    qoi[3 * s + 1] = (qmask & 2) ? q_pt : 0.0;
    qoi[3 * s + 2] = (qmask & 4) ? q_l2 : 0.0;
    int st = 0;
    if (!(fabs(q_out) < 1e300 && fabs(q_pt) < 1e300 && fabs(q_l2) < 1e300))
        st = CE_ERR_NONFINITE;
    else if (!(sc.orr[s] <= rtol2 * sc.orr0[s]))
        st = CE_ERR_NOT_CONVERGED;
    if (status_out) status_out[s] = st;
    if (iters_out) iters_out[s] = sc.iters[s];
    if (st != 0) atomicAdd(&misc[0], 1);
    atomicMax(&misc[1], sc.iters[s]);
    atomicAdd(&misc[2], sc.iters[s]);
}

// ---------------------------------------------------------------- driver
struct Solver3 {
    cudaStream_t st = nullptr;
    int count = 0, NL = 0;
    int n[MAXLEV3];
    long long V[MAXLEV3];
    float *gx[MAXLEV3] = {}, *gy[MAXLEV3] = {}, *gz[MAXLEV3] = {}, *b[MAXLEV3] = {},
          *z[MAXLEV3] = {};
    __half *hx[MAXLEV3] = {}, *hy[MAXLEV3] = {}, *hz[MAXLEV3] = {};   // multigrid copies
    float *res = nullptr, *p = nullptr, *q = nullptr, *d = nullptr;
    float *glx = nullptr, *gly = nullptr, *glz = nullptr;   // lo parts of the level-0 conductances
    float2 *uf = nullptr;                                    // u as float-float
    double *u = nullptr;                                     // u in FP64 for the QoIs
    double *part = nullptr, *part2 = nullptr, *sdbl = nullptr;
    int *sint = nullptr;
    Scal3 sc{};
    int nblk0 = 0;
    std::vector<void *> owned;

    template <typename T>
    int alloc(T **ptr, size_t cnt) {
        int rc = sce_alloc_t(ptr, cnt, st);
        if (rc == CE_OK) owned.push_back(*ptr);
        return rc;
    }
    ~Solver3() {
        for (void *ptr : owned) sce_free(ptr, st);
    }
    dim3 grid(int L) const { return dim3((unsigned)((V[L] + EPB3 - 1) / EPB3), count); }
    double vb(int L, double per) const { return (double)count * V[L] * per; }

    int init(int n0, int cnt) {
        count = cnt;
        NL = 0;
        for (int m = n0; m >= 2; m >>= 1) {
            n[NL] = m;
            V[NL] = (long long)(m + 1) * (m + 1) * (m + 1);
            ++NL;
        }
        for (int L = 0; L < NL; ++L) {
            const size_t c = (size_t)count * V[L];
            SCE_TRY(alloc(&gx[L], c));
            SCE_TRY(alloc(&gy[L], c));
            SCE_TRY(alloc(&gz[L], c));
            SCE_TRY(alloc(&b[L], c));
            SCE_TRY(alloc(&z[L], c));
            SCE_TRY(alloc(&hx[L], c));
            SCE_TRY(alloc(&hy[L], c));
            SCE_TRY(alloc(&hz[L], c));
        }
        const size_t c0 = (size_t)count * V[0];
        SCE_TRY(alloc(&res, c0));
        SCE_TRY(alloc(&p, c0));
        SCE_TRY(alloc(&q, c0));
        SCE_TRY(alloc(&d, c0));
        SCE_TRY(alloc(&glx, c0));
        SCE_TRY(alloc(&gly, c0));
        SCE_TRY(alloc(&glz, c0));
        SCE_TRY(alloc(&uf, c0));
        SCE_TRY(alloc(&u, c0));
        nblk0 = (int)((V[0] + EPB3 - 1) / EPB3);
        SCE_TRY(alloc(&part, (size_t)count * nblk0));
        SCE_TRY(alloc(&part2, (size_t)count * nblk0));
        SCE_TRY(alloc(&sdbl, (size_t)count * 8));
        SCE_TRY(alloc(&sint, (size_t)count * 4 + 4));
        sc.rz = sdbl;
        sc.pq = sdbl + count;
        sc.rr = sdbl + 2 * count;
        sc.alpha = sdbl + 3 * count;
        sc.beta = sdbl + 4 * count;
        sc.orr = sdbl + 5 * count;
        sc.orr0 = sdbl + 6 * count;
        sc.thr = sdbl + 7 * count;
        sc.act_out = sint;
        sc.act_in = sint + count;
        sc.iters = sint + 2 * count;
        sc.counter = sint + 4 * count;
        // vertices the kernels never write (Dirichlet planes of z and q) stay 0
        for (int L = 0; L < NL; ++L)
            SCE_CUDA(cudaMemsetAsync(z[L], 0, (size_t)count * V[L] * sizeof(float), st));
        SCE_CUDA(cudaMemsetAsync(q, 0, c0 * sizeof(float), st));
        SCE_CUDA(cudaMemsetAsync(sdbl, 0, (size_t)count * 8 * sizeof(double), st));
        SCE_CUDA(cudaMemsetAsync(sint, 0, ((size_t)count * 4 + 4) * sizeof(int), st));
        return CE_OK;
    }

    // nb = partials per sample of the producing kernel (-1: nblk0)
    void reduce(int mode, const int *act, double rtol2 = 0.0, double in_rel2 = 0.0, int nb = -1) {
        if (nb < 0) nb = nblk0;
        SceProf pr(KP_REDUCE, st, (double)count * nb * 8.0);
        reduce3_kernel<<<(count * 32 + 255) / 256, 256, 0, st>>>(part, nb, count, mode, sc, act,
                                                                 rtol2, in_rel2);
    }

    // row-structured launch: 2^lt threads per row of the w-wide grid
    dim3 rgrid(int w, int lt) const {
        const int rpb = 256 >> lt;
        return dim3((unsigned)((w * w + rpb - 1) / rpb), count);
    }

    int read_counter(int *host) {
        SCE_CUDA(cudaMemcpyAsync(host, sc.counter, sizeof(int), cudaMemcpyDeviceToHost, st));
        SCE_CUDA(cudaStreamSynchronize(st));
        return CE_OK;
    }

    // z[0] = M^-1 b[0] for the samples with act set
    // z[0] = M^-1 b[0] for the samples with act set
    void vcycle(const int *act) {
        if (NL == 1) cudaMemsetAsync(z[0], 0, (size_t)count * V[0] * sizeof(float), st);
        for (int L = 0; L < NL - 1; ++L) {
            const int w = n[L] + 1, lt = ilog2(n[L]);
            {
                SceProf pr(KP_SMOOTH3, st, vb(L, 2 * 6.0 + 3 * 4.0 + 2 * 4.0));
                smooth3_kernel<__half, true><<<rgrid(w, lt - 1), 256, 0, st>>>(
                    hx[L], hy[L], hz[L], b[L], z[L], n[L], lt - 1, 0, act);
                smooth3_kernel<__half, false><<<rgrid(w, lt - 1), 256, 0, st>>>(
                    hx[L], hy[L], hz[L], b[L], z[L], n[L], lt - 1, 1, act);
            }
            {
                SceProf pr(KP_RESID3, st, vb(L, 6.0 + 3 * 4.0));
                resid3_kernel<__half><<<rgrid(w, lt), 256, 0, st>>>(hx[L], hy[L], hz[L], b[L], z[L],
                                                                    res, n[L], lt, act);
            }
            {
                SceProf pr(KP_RESTRICT3, st, vb(L, 4.0) + vb(L + 1, 4.0));
                restrict3_kernel<<<rgrid(n[L + 1] + 1, lt - 1), 256, 0, st>>>(res, n[L], b[L + 1],
                                                                             lt - 1, act);
            }
        }
        {
            const int L = NL - 1;
            SceProf pr(KP_COARSEST, st, vb(L, 5 * 4.0));
            coarsest3_kernel<<<(count + 127) / 128, 128, 0, st>>>(gx[L], gy[L], gz[L], b[L], z[L],
                                                                   count, act);
        }
        for (int L = NL - 2; L >= 0; --L) {
            const int w = n[L] + 1, lt = ilog2(n[L]);
            {
                SceProf pr(KP_PROLONG3, st, vb(L, 8.0) + vb(L + 1, 4.0));
                prolong3_kernel<<<rgrid(w, lt), 256, 0, st>>>(z[L + 1], n[L + 1], z[L], lt, act);
            }
            SceProf pr(KP_SMOOTH3, st, vb(L, 2 * (6.0 + 3 * 4.0)));
            smooth3_kernel<__half, false><<<rgrid(w, lt - 1), 256, 0, st>>>(
                hx[L], hy[L], hz[L], b[L], z[L], n[L], lt - 1, 1, act);
            smooth3_kernel<__half, false><<<rgrid(w, lt - 1), 256, 0, st>>>(
                hx[L], hy[L], hz[L], b[L], z[L], n[L], lt - 1, 0, act);
        }
    }
};

// u_init: device double[count*(n+1)^3] or NULL (the lifting): the first
// iterate; the convergence test stays relative to the lifting's residual
int solve3(const darcy_problem *pr, const float *k, int count, double *qoi, int *iters,
           int *status, double *u_out, cudaStream_t st, int *misc_out, int qmask,
           const double *u_init) {
    Solver3 S;
    S.st = st;
    SCE_TRY(S.init(pr->n, count));
    const int n0 = pr->n;
    const dim3 g0 = S.grid(0);
    const long long V0 = S.V[0];
    {
        SceProf pf(KP_COND3, st, S.vb(0, 4.0 + 3 * 12.0));
        cond3_kernel<<<g0, TPB3, 0, st>>>(k, n0, S.gx[0], S.gy[0], S.gz[0], S.glx, S.gly, S.glz);
        const long long tot = (long long)count * V0;
        half3_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 1 << 20), 256, 0, st>>>(
            S.gx[0], S.gy[0], S.gz[0], tot, S.hx[0], S.hy[0], S.hz[0]);
    }
    for (int L = 1; L < S.NL; ++L) {
        SceProf pf(KP_COARSEN, st, S.vb(L - 1, 12.0) + S.vb(L, 12.0));
        coarsen3_kernel<<<S.grid(L), TPB3, 0, st>>>(S.gx[L - 1], S.gy[L - 1], S.gz[L - 1], S.n[L - 1],
                                                    S.gx[L], S.gy[L], S.gz[L], S.hx[L], S.hy[L],
                                                    S.hz[L]);
    }
    lift3_kernel<<<g0, TPB3, 0, st>>>(S.uf, n0);
    const Outer3 ost{S.gx[0], S.gy[0], S.gz[0], S.glx, S.gly, S.glz, S.uf};
    SCE_CUDA(cudaGetLastError());

    const double h = 1.0 / (double)n0;
    const double fh2 = pr->f * h * h;
    const double rtol2 = pr->rtol * pr->rtol;
    const double in_rel2 = 1e-10;   // inner target: relative drop 1e-5
    const int maxit = pr->maxit > 0 ? pr->maxit : 1000;
    const int inner_max = 40, check_every = 4;

    auto outer_residual = [&](const int *act, int mode) -> int {
        {
            SceProf pf(KP_OUTER3, st, S.vb(0, 4 * 8.0 + 4.0));
            outer_residual3_kernel<<<g0, TPB3, 0, st>>>(ost, n0, fh2, S.b[0], S.part, S.nblk0,
                                                        act);
        }
        SCE_CUDA(cudaMemsetAsync(S.sc.counter, 0, sizeof(int), st));
        S.reduce(mode, act, rtol2, in_rel2);
        SCE_CUDA(cudaGetLastError());
        return CE_OK;
    };
    SCE_TRY(outer_residual(nullptr, R3_ORR0));
    if (u_init) {
        const long long tot = (long long)count * V0;
        set_u3_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 1 << 20), 256, 0, st>>>(
            S.uf, u_init, tot);
        SCE_TRY(outer_residual(S.sc.act_out, R3_ORR));
    }
    int n_act = 0;
    SCE_TRY(S.read_counter(&n_act));
    int total_inner = 0;
    for (int outer = 0; outer < 64 && n_act > 0 && total_inner < maxit; ++outer) {
        SCE_CUDA(cudaMemsetAsync(S.d, 0, (size_t)count * V0 * sizeof(float), st));
        S.vcycle(S.sc.act_in);
        {
            SceProf pf(KP_DOT, st, S.vb(0, 8.0));
            dot3_kernel<<<g0, TPB3, 0, st>>>(S.b[0], S.z[0], V0, S.part, S.nblk0, S.sc.act_in);
        }
        {
            SceProf pf(KP_VEC3, st, S.vb(0, 8.0));
            pupdate3_kernel<<<g0, TPB3, 0, st>>>(S.p, S.z[0], S.sc.beta, V0, 1, S.sc.act_in);
        }
        S.reduce(R3_RZ0, S.sc.act_in);
        int in_act = n_act;
        for (int it = 0; it < inner_max && in_act > 0 && total_inner < maxit;) {
            {
                SceProf pf(KP_SPMV3, st, S.vb(0, 5 * 4.0));
                spmv_dot3_kernel<<<g0, TPB3, 0, st>>>(S.gx[0], S.gy[0], S.gz[0], S.p, S.q, n0,
                                                      S.part, S.nblk0, S.sc.act_in);
            }
            S.reduce(R3_ALPHA, S.sc.act_in);
            {
                SceProf pf(KP_VEC3, st, S.vb(0, 6 * 4.0));
                axpy2_3_kernel<<<g0, TPB3, 0, st>>>(S.d, S.b[0], S.p, S.q, S.sc.alpha, V0, S.part,
                                                    S.nblk0, S.sc.act_in);
            }
            SCE_CUDA(cudaMemsetAsync(S.sc.counter, 0, sizeof(int), st));
            S.reduce(R3_RR, S.sc.act_in);
            ++total_inner;
            ++it;
            if (it % check_every == 0) {
                SCE_TRY(S.read_counter(&in_act));
                if (in_act == 0) break;
            }
            S.vcycle(S.sc.act_in);
            {
                SceProf pf(KP_DOT, st, S.vb(0, 8.0));
                dot3_kernel<<<g0, TPB3, 0, st>>>(S.b[0], S.z[0], V0, S.part, S.nblk0, S.sc.act_in);
            }
            S.reduce(R3_BETA, S.sc.act_in);
            {
                SceProf pf(KP_VEC3, st, S.vb(0, 3 * 4.0));
                pupdate3_kernel<<<g0, TPB3, 0, st>>>(S.p, S.z[0], S.sc.beta, V0, 0, S.sc.act_in);
            }
        }
        SCE_CUDA(cudaGetLastError());
        {
            SceProf pf(KP_OUTER3, st, S.vb(0, 2 * 8.0 + 4.0));
            outer_update3_kernel<<<g0, TPB3, 0, st>>>(S.uf, S.d, n0, S.sc.act_out);
        }
        SCE_TRY(outer_residual(S.sc.act_out, R3_ORR));
        SCE_TRY(S.read_counter(&n_act));
    }

    {
        const long long tot = (long long)count * V0;
        u_to_double3_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 1 << 20), 256, 0,
                              st>>>(S.uf, tot, S.u);
    }
    const bool grid_qoi = (qmask & 5) != 0;   // outflow and L2 norm need a pass over the grid
    if (grid_qoi) {
        SceProf pf(KP_QOI, st, S.vb(0, 16.0));
        qoi3_partial_kernel<<<g0, TPB3, 0, st>>>(S.gx[0], S.glx, S.u, n0, fh2, S.part, S.part2,
                                                 S.nblk0);
    }
    int *misc = S.sint + 4 * count + 1;   // [failed, max iters, total iters]
    SCE_CUDA(cudaMemsetAsync(misc, 0, 3 * sizeof(int), st));
    qoi3_final_kernel<<<(count * 32 + 255) / 256, 256, 0, st>>>(
        grid_qoi ? S.part : nullptr, grid_qoi ? S.part2 : nullptr, S.nblk0, count, S.u, n0, S.sc,
        rtol2, qoi, iters, status, misc, qmask);
    SCE_CUDA(cudaGetLastError());
    if (u_out)
        SCE_CUDA(cudaMemcpyAsync(u_out, S.u, (size_t)count * V0 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
    int hm[3] = {0, 0, 0};
    SCE_CUDA(cudaMemcpyAsync(hm, misc, sizeof(hm), cudaMemcpyDeviceToHost, st));
    SCE_CUDA(cudaStreamSynchronize(st));
    if (misc_out) {
        misc_out[0] = hm[0];
        misc_out[1] = hm[1];
        misc_out[2] = hm[2];
    }
    return hm[0] > 0 ? CE_ERR_NOT_CONVERGED : CE_OK;
}

// samples per solve call: device memory bounded to about 8 GB
int chunk3(int n) {
    const double V = (double)(n + 1) * (n + 1) * (n + 1);
    const double per = V * (9 * 4.0 + 4 * 8.0) * 1.15 + 1024;
    return (int)std::max(1.0, std::min(65535.0, std::floor(8e9 / per)));
}

int solve3_batched(const darcy_problem *p, const float *k, int count, double *qoi, int *iters,
                   int *status, double *u_out, cudaStream_t st, int *misc_out, int qmask,
                   const double *u_init = nullptr) {
    const int chunk = chunk3(p->n);
    const long long V = (long long)(p->n + 1) * (p->n + 1) * (p->n + 1);
    int worst = CE_OK;
    int tot[3] = {0, 0, 0};
    for (int c0 = 0; c0 < count; c0 += chunk) {
        const int cn = std::min(chunk, count - c0);
        int m[3] = {0, 0, 0};
        const int rc = solve3(p, k + (size_t)c0 * V, cn, qoi + 3 * (size_t)c0,
                              iters ? iters + c0 : nullptr, status ? status + c0 : nullptr,
                              u_out ? u_out + (size_t)c0 * V : nullptr, st, m, qmask,
                              u_init ? u_init + (size_t)c0 * V : nullptr);
        if (rc != CE_OK && rc != CE_ERR_NOT_CONVERGED) return rc;
        if (rc != CE_OK) worst = rc;
        tot[0] += m[0];
        tot[1] = std::max(tot[1], m[1]);
        tot[2] += m[2];
    }
    if (misc_out) {
        misc_out[0] = tot[0];
        misc_out[1] = tot[1];
        misc_out[2] = tot[2];
    }
    return worst;
}

}  // namespace

extern "C" int darcy3_solve_batch(const darcy_problem *p, const float *k, int count, double *qoi,
                                  int *iters, int *status, double *u_out, void *stream) {
    if (!p || !k || !qoi || count < 0) return CE_ERR_INVALID_ARG;
    if (!is_pow2(p->n) || p->n < 2 || p->n > 256 || p->precision != 32 || !(p->rtol > 0))
        return CE_ERR_INVALID_ARG;
    if (count == 0) return CE_OK;
    return solve3_batched(p, k, count, qoi, iters, status, u_out, as_stream(stream), nullptr, 7);
}

extern "C" int mlmc3_level_estimate(ce3_embedding_t e, const darcy_problem *p, uint64_t seed,
                                    uint32_t level, uint64_t first_sample, int count,
                                    int qoi_index, mlmc_level_sums *out, double *Y,
                                    void *stream) {
    if (!e || !p || !out || count < 0 || qoi_index < 0 || qoi_index > 2) return CE_ERR_INVALID_ARG;
    ce_embedding_info info;
    SCE_TRY(ce3_get_info(e, &info));
    if (p->n != info.n || p->precision != 32 || !(p->rtol > 0)) return CE_ERR_INVALID_ARG;
    if (level > 0 && p->n < 4) return CE_ERR_INVALID_ARG;
    *out = mlmc_level_sums{};
    if (count == 0) return CE_OK;
    cudaStream_t st = as_stream(stream);
    const int n = p->n, nc = n / 2;
    const long long Vf = (long long)(n + 1) * (n + 1) * (n + 1);
    const long long Vc = (long long)(nc + 1) * (nc + 1) * (nc + 1);
    const int chunk = std::min(count, std::max(1, chunk3(n) / 2));
    float *kf = nullptr, *kc = nullptr;
    double *qf = nullptr, *qc = nullptr, *ucs = nullptr, *uf0 = nullptr;
    int rc = sce_alloc_t(&kf, (size_t)chunk * Vf, st);
    if (rc == CE_OK && level > 0) rc = sce_alloc_t(&kc, (size_t)chunk * Vc, st);
    // nested iteration: the coarse solve first, its prolonged solution the
    // fine solve's first iterate
    if (rc == CE_OK && level > 0) rc = sce_alloc_t(&ucs, (size_t)chunk * Vc, st);
    if (rc == CE_OK && level > 0) rc = sce_alloc_t(&uf0, (size_t)chunk * Vf, st);
    if (rc == CE_OK) rc = sce_alloc_t(&qf, (size_t)chunk * 3, st);
    if (rc == CE_OK && level > 0) rc = sce_alloc_t(&qc, (size_t)chunk * 3, st);
    std::vector<double> hf((size_t)chunk * 3), hc((size_t)chunk * 3), hy(chunk);
    darcy_problem pc = *p;
    pc.n = nc;
    int worst = CE_OK;
    for (int c0 = 0; c0 < count && rc == CE_OK; c0 += chunk) {
        const int cn = std::min(chunk, count - c0);
        rc = ce3_sample_batch(e, seed, level, first_sample + c0, cn, kf, level > 0 ? kc : nullptr,
                              stream);
        int m[3] = {0, 0, 0};
        if (rc == CE_OK && level > 0) {
            rc = solve3_batched(&pc, kc, cn, qc, nullptr, nullptr, ucs, st, m, 1 << qoi_index);
            out->n_failed += m[0];
            out->max_iters = std::max(out->max_iters, m[1]);
            out->total_iters += m[2];
            if (rc == CE_ERR_NOT_CONVERGED) {
                worst = rc;
                rc = CE_OK;
            }
            if (rc == CE_OK) {
                const long long tot = (long long)cn * Vf;
                prolong_u3_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 1 << 20), 256,
                                    0, st>>>(ucs, nc, cn, uf0);
                if (cudaGetLastError() != cudaSuccess) rc = CE_ERR_CUDA;
            }
        }
        if (rc == CE_OK) {
            rc = solve3_batched(p, kf, cn, qf, nullptr, nullptr, nullptr, st, m, 1 << qoi_index,
                                level > 0 ? uf0 : nullptr);
            out->n_failed += m[0];
            out->max_iters = std::max(out->max_iters, m[1]);
            out->total_iters += m[2];
            if (rc == CE_ERR_NOT_CONVERGED) {
                worst = rc;
                rc = CE_OK;
            }
        }
        if (rc != CE_OK) break;
        if (cudaMemcpyAsync(hf.data(), qf, (size_t)cn * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            (level > 0 && cudaMemcpyAsync(hc.data(), qc, (size_t)cn * 3 * sizeof(double),
                                          cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = CE_ERR_CUDA;
            break;
        }
        // level sums in sample order (Eq. (3.5))
        for (int i = 0; i < cn; ++i) {
            const double Qf = hf[3 * (size_t)i + qoi_index];
            const double Yi = level > 0 ? Qf - hc[3 * (size_t)i + qoi_index] : Qf;
            hy[i] = Yi;
            out->sumY += Yi;
            out->sumY2 += Yi * Yi;
            out->sumQf += Qf;
            out->sumQf2 += Qf * Qf;
        }
        out->N += cn;
        if (Y && cudaMemcpyAsync(Y + c0, hy.data(), (size_t)cn * sizeof(double),
                                 cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = CE_ERR_CUDA;
            break;
        }
        if (Y && cudaStreamSynchronize(st) != cudaSuccess) {
            rc = CE_ERR_CUDA;
            break;
        }
    }
    sce_free(kf, st);
    sce_free(kc, st);
    sce_free(qf, st);
    sce_free(qc, st);
    sce_free(ucs, st);
    sce_free(uf0, st);
    cudaStreamSynchronize(st);
    return rc != CE_OK ? rc : worst;
}

extern "C" int mlmc3_estimate_levels(const darcy_problem *p, uint64_t seed, int qoi_index,
                                     mlmc3_level_task *tasks, int ntasks, int max_concurrency,
                                     void *stream) {
    if (!p || ntasks < 0 || (ntasks > 0 && !tasks) || qoi_index < 0 || qoi_index > 2 ||
        p->precision != 32 || !(p->rtol > 0))
        return CE_ERR_INVALID_ARG;
    for (int i = 0; i < ntasks; ++i)
        if (!tasks[i].emb || tasks[i].count < 0) return CE_ERR_INVALID_ARG;
    for (int i = 0; i < ntasks; ++i) {
        tasks[i].sums = mlmc_level_sums{};
        tasks[i].status = CE_OK;
    }
    const cudaStream_t st = as_stream(stream);
    auto run = [&](int i, cudaStream_t s) {
        ce_embedding_info info;
        int rc = ce3_get_info(tasks[i].emb, &info);
        if (rc == CE_OK) {
            darcy_problem q = *p;
            q.n = info.n;
            rc = mlmc3_level_estimate(tasks[i].emb, &q, seed, tasks[i].level,
                                      tasks[i].first_sample, tasks[i].count, qoi_index,
                                      &tasks[i].sums, tasks[i].Y, (void *)s);
        }
        tasks[i].status = rc;
    };
    auto combine = [&]() {
        int worst = CE_OK;
        for (int i = 0; i < ntasks; ++i) {
            const int r = tasks[i].status;
            if (r != CE_OK && r != CE_ERR_NOT_CONVERGED) return r;
            if (r == CE_ERR_NOT_CONVERGED) worst = r;
        }
        return worst;
    };
    if (max_concurrency <= 1 || ntasks == 0) {
        for (int i = 0; i < ntasks; ++i) {
            run(i, st);
            if (tasks[i].status != CE_OK && tasks[i].status != CE_ERR_NOT_CONVERGED) break;
        }
        return combine();
    }
    int dev = 0;
    SCE_CUDA(cudaGetDevice(&dev));
    std::vector<cudaStream_t> ss((size_t)ntasks, nullptr);
    std::vector<cudaEvent_t> evs;
    auto release = [&]() {
        for (cudaStream_t s : ss)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    };
    auto new_event = [&](cudaEvent_t *ev) {
        const cudaError_t err = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (err == cudaSuccess) evs.push_back(*ev);
        return err;
    };
    cudaEvent_t ev0;
    if (new_event(&ev0) != cudaSuccess || cudaEventRecord(ev0, st) != cudaSuccess) {
        release();
        return CE_ERR_CUDA;
    }
    for (int i = 0; i < ntasks; ++i) {
        if (cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamWaitEvent(ss[i], ev0, 0) != cudaSuccess) {
            release();
            return CE_ERR_CUDA;
        }
    }
    // largest levels first: they bound the makespan
    std::vector<int> order(ntasks);
    std::vector<double> work(ntasks, 0.0);
    for (int i = 0; i < ntasks; ++i) {
        order[i] = i;
        ce_embedding_info info;
        if (ce3_get_info(tasks[i].emb, &info) == CE_OK)
            work[i] = (double)tasks[i].count * (info.n + 1.0) * (info.n + 1.0) * (info.n + 1.0);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    std::atomic<int> next{0};
    std::mutex err_mu;
    std::string err_text;
    auto worker = [&]() {
        if (cudaSetDevice(dev) != cudaSuccess) return;
        for (int k; (k = next.fetch_add(1)) < ntasks;) {
            const int i = order[k];
            run(i, ss[i]);
            if (tasks[i].status != CE_OK && tasks[i].status != CE_ERR_NOT_CONVERGED) {
                std::lock_guard<std::mutex> lk(err_mu);
                if (err_text.empty()) err_text = sce_last_error();
            }
        }
    };
    const int nthreads = std::min(max_concurrency, ntasks);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(worker);
    for (std::thread &t : pool) t.join();
    if (!err_text.empty()) sce_set_last_error_text(err_text.c_str());
    for (cudaStream_t s : ss) {
        cudaEvent_t ev;
        if (new_event(&ev) != cudaSuccess || cudaEventRecord(ev, s) != cudaSuccess ||
            cudaStreamWaitEvent(st, ev, 0) != cudaSuccess) {
            release();
            return CE_ERR_CUDA;
        }
    }
    release();
    return combine();
}

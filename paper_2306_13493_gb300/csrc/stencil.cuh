// Per-vertex pieces of the five-point P1 operator and of the multigrid cycle,
// shared by the grid-wide batched kernels and the one-block-per-sample solver.
// All functions take the base pointer of one sample's array on an n-cell grid
// (row-major, x-fastest, n+1 vertices per row); they work on global or shared
// memory.  w (or wf / wc for the fine / coarse grid): the arrays' row pitch,
// 0 for the dense layout (n + 1); padded shared-memory levels pass n + 2.
#pragma once

#include "ff.cuh"

namespace sce {

// Edge conductances at vertex (i, j) from the vertex values of k, in FP64:
//   gx = cx(i,j) = 1/2 [kbar_T1(i,j) + kbar_T2(i,j-1)]   (0 if i == n)
//   gy = cy(i,j) = 1/2 [kbar_T2(i,j) + kbar_T1(i-1,j)]   (0 if j == n)
// T1(a,b) = {(a,b),(a+1,b),(a+1,b+1)}, T2(a,b) = {(a,b),(a,b+1),(a+1,b+1)}.
// The sums are of at most six vertex values (exact in FP64 for FP32 k) and
// are scaled once by 1/6 (= 1/2 * 1/3): no FP64 division.
template <typename Tk>
__device__ __forceinline__ void cond_at(const Tk *ks, int i, int j, int n, double *gx,
                                        double *gy) {
    const int w = n + 1, v = j * w + i;
    const double a = (double)ks[v];                                   // k(i, j)
    const double b = i < n ? (double)ks[v + 1] : 0.0;                 // k(i+1, j)
    const double e = j < n ? (double)ks[v + w] : 0.0;                 // k(i, j+1)
    const double c = (i < n && j < n) ? (double)ks[v + w + 1] : 0.0; // k(i+1, j+1)
    double x = 0.0, y = 0.0;
    if (i < n) {
        const double ab = a + b;                                      // shared by T1, T2
        if (j < n) x = ab + c;                                        // T1(i, j)
        if (j > 0) x += ab + (double)ks[v - w];                       // T2(i, j-1)
        x *= (1.0 / 6.0);
    }
    if (j < n) {
        const double ae = a + e;
        if (i < n) y = ae + c;                                        // T2(i, j)
        if (i > 0) y += ae + (double)ks[v - 1];                       // T1(i-1, j)
        y *= (1.0 / 6.0);
    }
    *gx = x;
    *gy = y;
}

// 1/6 as a float-float (nearest float, and the float nearest to the rest)
__device__ __forceinline__ ff ff_sixth() { return {0x1.555556p-3f, -0x1.555556p-28f}; }

// cond_at in float-float from FP32 k: the same sums of at most six vertex
// values and one scaling by 1/6.  The two triangles of an edge share the two
// vertex values a, b of the edge itself, so an interior edge sums to
// 2 (a + b) + c + d: TwoSum(a, b), an exact doubling, and two float-float +
// float additions (positive terms: no cancellation, relative error ~2^-47).
__device__ __forceinline__ void cond_at_ff(const float *ks, int i, int j, int n, ff *gx, ff *gy) {
    const int w = n + 1, v = j * w + i;
    const float a = ks[v];
    ff x = {0.0f, 0.0f}, y = {0.0f, 0.0f};
    if (i < n) {
        const float b = ks[v + 1];                       // k(i+1, j)
        x = two_sum(a, b);
        if (j > 0 && j < n) x = {2.0f * x.hi, 2.0f * x.lo};
        if (j < n) x = ff_add_f(x, ks[v + w + 1]);      // T1(i, j): k(i+1, j+1)
        if (j > 0) x = ff_add_f(x, ks[v - w]);          // T2(i, j-1): k(i, j-1)
        x = ff_mul(x, ff_sixth());
    }
    if (j < n) {
        const float e = ks[v + w];                       // k(i, j+1)
        y = two_sum(a, e);
        if (i > 0 && i < n) y = {2.0f * y.hi, 2.0f * y.lo};
        if (i < n) y = ff_add_f(y, ks[v + w + 1]);      // T2(i, j): k(i+1, j+1)
        if (i > 0) y = ff_add_f(y, ks[v - 1]);          // T1(i-1, j): k(i-1, j)
        y = ff_mul(y, ff_sixth());
    }
    *gx = x;
    *gy = y;
}

// F - (A u)(i, j) at an unknown vertex, rounded once to FP32: the residual of
// the float-float refinement.  u as (hi, lo) pairs, conductances hi (cx, cy) +
// lo (cxl, cyl), F a float-float.  For every edge to a neighbour nb:
//   u_c - u_nb = TwoSum of the hi parts (exact) + the difference of the lo
//                parts (two FP32 roundings of terms below ulp(u));
//   c (u_c - u_nb) = TwoProduct of the hi parts (exact) + the cross terms
//                c_hi * d_lo + c_lo * d_hi (fused, the c_lo * d_lo term is
//                below 2^-48 of the product and dropped);
// F.hi minus the four product hi parts is summed by a cascade of TwoSums, and
// their rounding errors together with every low-order term in plain FP32
// (Algorithm Sum2 of Ogita, Rump and Oishi, "Accurate sum and dot product",
// 2005); the two sums are added once at the end.  The error stays of the
// order 2^-48 of |u| and of the products, the resolution of the float-float
// operands themselves, at about 80 FP32 operations against ~190 for composing
// float-float subtractions, products and sums.
__device__ __forceinline__ float resid_at_ff(ff F, const float *cx, const float *cxl,
                                             const float *cy, const float *cyl, const float2 *u,
                                             int i, int j, int n, int w = 0) {
    if (w <= 0) w = n + 1;
    const int v = j * w + i;
    const float2 uc = u[v];
    float p = F.hi, sig = F.lo;
    auto edge = [&](float ch, float cl, float2 un) {
        const ff d = two_sum(uc.x, -un.x);
        const float dl = __fadd_rn(d.lo, __fsub_rn(uc.y, un.y));
        const ff pr = two_prod(ch, d.hi);
        const float pl = __fmaf_rn(cl, d.hi, __fmaf_rn(ch, dl, pr.lo));
        const ff t = two_sum(p, -pr.hi);
        p = t.hi;
        sig = __fadd_rn(sig, __fsub_rn(t.lo, pl));
    };
    edge(cx[v - 1], cxl[v - 1], u[v - 1]);
    edge(cx[v], cxl[v], u[v + 1]);
    if (j > 0) edge(cy[v - w], cyl[v - w], u[v - w]);
    if (j < n) edge(cy[v], cyl[v], u[v + w]);
    return __fadd_rn(p, sig);
}

// Series conductance a b / (a + b) of two edges.  It only enters the
// coarse operators of the multigrid preconditioner, which has to be a fixed
// symmetric operation, not an exact one (the refinement removes its
// rounding): FP32 uses the fast single-precision division, as the smoothers
// do; FP64 keeps the exact division.
template <typename T>
__device__ __forceinline__ T series_cond(T a, T b) {
    const T t = a + b;
    if constexpr (sizeof(T) == 4) return t > T(0) ? __fdividef(a * b, t) : T(0);
    else return t > T(0) ? a * b / t : T(0);
}

// Coarse conductances at coarse vertex (I, J): a coarse edge spans two fine
// edges in series and stands for the fine lines 2J (weight 1), 2J +- 1 (1/2).
// Computed in the working precision T of the hierarchy.
template <typename T>
__device__ __forceinline__ void coarsen_at(const T *ax, const T *ay, int nf, int I, int J, T *gx,
                                           T *gy, int wf = 0) {
    const int nc = nf / 2;
    if (wf <= 0) wf = nf + 1;
    T x = T(0), y = T(0);
    if (I < nc) {
        auto S = [&](int j) { return series_cond(ax[j * wf + 2 * I], ax[j * wf + 2 * I + 1]); };
        x = S(2 * J);
        if (J > 0) x += T(0.5) * S(2 * J - 1);
        if (J < nc) x += T(0.5) * S(2 * J + 1);
    }
    if (J < nc) {
        auto S = [&](int i) { return series_cond(ay[(2 * J) * wf + i], ay[(2 * J + 1) * wf + i]); };
        y = S(2 * I);
        if (I > 0) y += T(0.5) * S(2 * I - 1);
        if (I < nc) y += T(0.5) * S(2 * I + 1);
    }
    *gx = x;
    *gy = y;
}

// (A p)(i,j) at an unknown vertex (1 <= i <= n-1).
template <typename T>
__device__ __forceinline__ T apply_at(const T *ax, const T *ay, const T *p, int i, int j, int n,
                                      int w = 0) {
    if (w <= 0) w = n + 1;
    const int v = j * w + i;
    const T pc = p[v];
    T a = ax[v - 1] * (pc - p[v - 1]) + ax[v] * (pc - p[v + 1]);
    if (j > 0) a += ay[v - w] * (pc - p[v - w]);
    if (j < n) a += ay[v] * (pc - p[v + w]);
    return a;
}

// b - A z at an unknown vertex.
template <typename T>
__device__ __forceinline__ T resid_at(const T *ax, const T *ay, const T *b, const T *z, int i,
                                      int j, int n, int w = 0) {
    if (w <= 0) w = n + 1;
    return b[j * w + i] - apply_at(ax, ay, z, i, j, n, w);
}

// Division in the smoothers: the fast single-precision form in FP32 (a
// smoother only has to be a fixed symmetric operation, the refinement removes
// its rounding), the correctly rounded one in FP64.
__device__ __forceinline__ float smooth_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double smooth_div(double a, double b) { return a / b; }

// Gauss-Seidel update of one unknown vertex.
template <typename T>
__device__ __forceinline__ void smooth_at(const T *ax, const T *ay, const T *b, T *z, int i, int j,
                                          int n, int w = 0) {
    if (w <= 0) w = n + 1;
    const int v = j * w + i;
    const T cw = ax[v - 1], ce = ax[v];
    const T cs = j > 0 ? ay[v - w] : T(0), cn = j < n ? ay[v] : T(0);
    T acc = b[v] + cw * z[v - 1] + ce * z[v + 1];
    if (j > 0) acc += cs * z[v - w];
    if (j < n) acc += cn * z[v + w];
    z[v] = smooth_div(acc, cw + ce + cs + cn);
}

// Full-weighting restriction (transpose of bilinear prolongation) of the
// fine residual to coarse unknown (I, J), 1 <= I <= nc-1, right after a
// black half-sweep: the residual then vanishes at the black vertices (each was
// just solved for with its red neighbours fixed), so of the 3 x 3 stencil
// only the red ones count -- the coarse vertex itself (weight 1) and its four
// diagonal neighbours (weight 1/4), as in the tiled kernels.
template <typename T>
__device__ __forceinline__ T restrict_at(const T *ax, const T *ay, const T *b, const T *z, int nf,
                                         int I, int J, int wf = 0) {
    T acc = resid_at(ax, ay, b, z, 2 * I, 2 * J, nf, wf);
    T d = T(0);
    for (int dj = -1; dj <= 1; dj += 2) {
        const int j = 2 * J + dj;
        if (j < 0 || j > nf) continue;
        d += resid_at(ax, ay, b, z, 2 * I - 1, j, nf, wf) +
             resid_at(ax, ay, b, z, 2 * I + 1, j, nf, wf);
    }
    return acc + T(0.25) * d;
}

// Bilinear prolongation of the coarse correction to fine vertex (i, j).
template <typename T>
__device__ __forceinline__ T prolong_at(const T *c, int nc, int i, int j, int wc = 0) {
    if (wc <= 0) wc = nc + 1;
    const int I = i >> 1, J = j >> 1;
    if (!(i & 1) && !(j & 1)) return c[J * wc + I];
    if ((i & 1) && !(j & 1)) return T(0.5) * (c[J * wc + I] + c[J * wc + I + 1]);
    if (!(i & 1) && (j & 1)) return T(0.5) * (c[J * wc + I] + c[(J + 1) * wc + I]);
    return T(0.25) * (c[J * wc + I] + c[J * wc + I + 1] + c[(J + 1) * wc + I] +
                      c[(J + 1) * wc + I + 1]);
}

// Exact solve on the 2-cell grid (unknowns (1, j), j = 0..2; tridiagonal in j).
template <typename T>
__device__ __forceinline__ void coarsest_solve(const T *ax, const T *ay, const T *b, T *z) {
    // Thomas algorithm in the working precision (one thread; FP64 division
    // runs at a small fraction of the FP32 rate on GB300 and this sits on the
    // critical path of every cycle)
    T d[3], r[3];
    for (int j = 0; j < 3; ++j) {
        const int v = j * 3 + 1;
        d[j] = ax[v - 1] + ax[v] + (j > 0 ? ay[v - 3] : T(0)) + (j < 2 ? ay[v] : T(0));
        r[j] = b[v];
    }
    const T o0 = -ay[1], o1 = -ay[4];
    const T c0 = o0 / d[0];
    const T r0 = r[0] / d[0];
    const T den1 = d[1] - o0 * c0;
    const T c1 = o1 / den1;
    const T r1 = (r[1] - o0 * r0) / den1;
    const T den2 = d[2] - o1 * c1;
    const T x2 = (r[2] - o1 * r1) / den2;
    const T x1 = r1 - c1 * x2;
    const T x0 = r0 - c0 * x1;
    z[1] = x0;
    z[4] = x1;
    z[7] = x2;
}

}  // namespace sce

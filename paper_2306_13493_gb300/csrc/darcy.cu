// Batched Darcy solver: Eq. (3.1) with P1 elements and nodal quadrature (§3.2).
//
// Discrete operator.  Each cell [a,a+1]x[b,b+1] of the n-cell grid is split by
// the diagonal (a,b)-(a+1,b+1) into T1 = {(a,b),(a+1,b),(a+1,b+1)} and
// T2 = {(a,b),(a,b+1),(a+1,b+1)}; k is averaged over each triangle's vertices.
// On these right triangles the P1 stiffness couples only the two legs, each
// with weight -1/2 kbar_T (the hypotenuse coupling vanishes), so the matrix is
// the five-point graph Laplacian with edge conductances
//   cx(i,j) = 1/2 [kbar_T1(i,j) + kbar_T2(i,j-1)]   edge (i,j)-(i+1,j)
//   cy(i,j) = 1/2 [kbar_T2(i,j) + kbar_T1(i-1,j)]   edge (i,j)-(i,j+1)
// (terms of triangles outside the grid dropped) and the load is
// F = f h^2/6 * (number of triangles at the vertex).  Dirichlet columns
// i = 0 (u = 1) and i = n (u = 0) are kept in the arrays and never updated.
//
// Solver.  u (nodal, Dirichlet values included) is improved by iterative
// refinement: r = F - A u in high precision; the correction equation A d = r
// is solved by CG preconditioned with one symmetric multigrid cycle: in FP32
// two red-black Gauss-Seidel sweeps before and two black-red sweeps after each
// coarse correction on the finest level and on the levels wider than 128
// cells, three on the coarser levels (the per-level counts keep the cycle
// symmetric); V(1,1) in FP64; full-weighting
// restriction = transpose of bilinear
// prolongation, coarse conductances by series/parallel edge averaging, exact
// tridiagonal solve on the 2-cell grid), in FP32 (precision 32) or FP64
// (precision 64); u += d.  High precision is FP64 on the FP64 path and
// float-float (ff.cuh: ~48 bits from FP32 operations, which GB300 runs ~64x
// faster than FP64 ones) on the mixed path: u, the conductances (hi = the
// FP32 operator of the inner solve, lo = its rounding error) and the residual.
// Batched over samples: grid.y = sample, every
// kernel skips samples whose flag is clear, and all reductions are
// two-stage in a fixed order (bit-reproducible).
//
// QoIs: outflow = sum_j cx(n-1,j) u(n-1,j) + f h/2 (the consistent flux
// -sum (A u - F) over x1 = 1); u(7/15,7/15) from the P1 interpolant;
// ||u_h||_L2^2 = sum_T |T|/12 [(u_a+u_b+u_c)^2 + u_a^2 + u_b^2 + u_c^2].
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "ff.cuh"
#include "mg_tiles.cuh"
#include "mg_v64.cuh"
#include "sce_internal.cuh"

using namespace sce;

namespace {

constexpr int MAXLEV = 14;
#ifndef SCE_TAIL_N
#define SCE_TAIL_N 32
#endif
constexpr int TAIL_N = SCE_TAIL_N;   // levels with n <= TAIL_N run in one block per sample

// Sweeps per side on the coarse levels of the FP32 cycle: on grids of 128
// cells or more, every level below the finest of at most MG_NU_COARSE_MAX cells takes
// SCE_MG_NU_COARSE sweeps (3 by default; 2 gives the uniform V(2,2) cycle).
// On the oscillatory fields the third sweep on those levels (all of them: on
// a subset it gains nothing) takes a solve at n = 128..512 from ~9.3 to ~8.4
// CG iterations for a few percent more work per cycle; on n = 64 grids it
// saved too little to pay for the extra barrier-bound sweeps of the fused
// n = 64 cycle's shared-memory levels.
constexpr int MG_NU_COARSE_MAX = 128;
int mg_nu_coarse() {
    const char *e = getenv("SCE_MG_NU_COARSE");
    return (e && atoi(e) == 2) ? 2 : 3;
}

// Window heights of the tiled multigrid kernels, per (precision, grid size),
// chosen by darcy_autotune_tiles; MG_SH where absent (SCE_TILE_SH forces one
// for every level).  Every height computes each vertex of a V-cycle
// identically; the per-tile r . z partial sums follow the tiling, so the
// solves take different rounding paths to the same stopping tolerance.
constexpr int kTileHeights[] = {16, 24, 32, 48, 64};
std::mutex g_tile_mu;
std::map<std::pair<int, int>, int> g_tile_sh;   // (sizeof T, n) -> window height

int tile_height_for(int tsize, int n) {
    if (const char *e = getenv("SCE_TILE_SH")) {
        const int v = atoi(e);
        for (int h : kTileHeights)
            if (h == v) return v;
    }
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile_sh.find({tsize, n});
    return it == g_tile_sh.end() ? MG_SH : it->second;
}

struct Launch {
    int tpb, vpt, epb, nblk;
    long long V;
};

static Launch launch_for(int n) {
    Launch L;
    L.V = (long long)(n + 1) * (n + 1);
#ifndef SCE_EPB
#define SCE_EPB 2048
#endif
    long long e = 1;
    while (e < L.V && e < SCE_EPB) e <<= 1;
    L.epb = (int)e;
    L.tpb = std::min(256, L.epb);
    L.vpt = L.epb / L.tpb;
    L.nblk = (int)((L.V + L.epb - 1) / L.epb);
    return L;
}

// FOR_VERT with a compile-time count VPT (> 0; unrolled, so the loads of all
// elements are in flight together) or the run-time count vpt (VPT == 0)
#define FOR_VERT_C(V, VPT, vpt)                                                        \
    _Pragma("unroll") for (int e_ = 0, v = blockIdx.x * (blockDim.x * ((VPT) ? (VPT) : (vpt))) + \
                                           threadIdx.x;                                \
                           e_ < ((VPT) ? (VPT) : (vpt)); ++e_, v += blockDim.x)        \
        if (v < (V))

// vertex loop of one block: v = blockIdx.x*epb + threadIdx.x + e*blockDim.x
#define FOR_VERT(V, vpt)                                                               \
    for (int e_ = 0, v = blockIdx.x * (blockDim.x * (vpt)) + threadIdx.x; e_ < (vpt);  \
         ++e_, v += blockDim.x)                                                        \
        if (v < (V))

// Row index of vertex v on a grid of width w without an integer division:
// floor(v / w) = (v * ceil(2^40 / w)) >> 40, exact whenever v w < 2^40 (every
// grid up to n = 4096; checked exhaustively for all widths on the host).
inline unsigned long long row_magic(int w) { return ((1ull << 40) + (unsigned)w - 1) / (unsigned)w; }
__device__ __forceinline__ int vrow(int v, unsigned long long m) {
    return (int)(((unsigned long long)(unsigned)v * m) >> 40);
}

template <typename T>
__device__ __forceinline__ T block_sum(T val, T *sh) {
    // fixed-order tree: warp shuffles then warp partials in order
    for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = val;
    __syncthreads();
    T tot = T(0);
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) tot += sh[i];
    }
    return tot;   // valid in thread 0
}

// ---------------------------------------------------------------- operator
// Conductances of the fine grid.  FP64 path (T = double): FP64.  Mixed path
// (T = float): float-float, hi to cx/cy (the operator of the FP32 inner
// solve and of the hierarchy), lo to cxl/cyl.
template <typename Tk, typename T, int VPT = 0>
__global__ void cond_kernel(const Tk *__restrict__ k, int n, int vpt, T *__restrict__ cx,
                            T *__restrict__ cy, float *__restrict__ cxl,
                            float *__restrict__ cyl, unsigned long long rdm) {
    const int s = blockIdx.y;
    const long long V = (long long)(n + 1) * (n + 1);
    const Tk *ks = k + s * V;
    const int w = n + 1;
    FOR_VERT_C(V, VPT, vpt) {
        const int j = vrow(v, rdm), i = v - j * w;
        if constexpr (sizeof(T) == 4 && sizeof(Tk) == 4) {
            ff gx, gy;
            cond_at_ff(ks, i, j, n, &gx, &gy);
            cx[s * V + v] = gx.hi;
            cy[s * V + v] = gy.hi;
            cxl[s * V + v] = gx.lo;
            cyl[s * V + v] = gy.lo;
        } else {
            double gx, gy;
            cond_at(ks, i, j, n, &gx, &gy);
            cx[s * V + v] = (T)gx;
            cy[s * V + v] = (T)gy;
        }
    }
}

template <typename T, int VPT = 0>
__global__ void coarsen_kernel(const T *__restrict__ cxf, const T *__restrict__ cyf, int nf,
                               int vpt, T *__restrict__ cxc, T *__restrict__ cyc,
                               unsigned long long rdm) {
    const int s = blockIdx.y;
    const int nc = nf / 2;
    const long long Vf = (long long)(nf + 1) * (nf + 1), Vc = (long long)(nc + 1) * (nc + 1);
    const T *ax = cxf + s * Vf, *ay = cyf + s * Vf;
    const int wc = nc + 1;
    FOR_VERT_C(Vc, VPT, vpt) {
        const int J = vrow(v, rdm), I = v - J * wc;
        T gx, gy;
        coarsen_at(ax, ay, nf, I, J, &gx, &gy);
        cxc[s * Vc + v] = gx;
        cyc[s * Vc + v] = gy;
    }
}

// ---------------------------------------------------------------- multigrid
// Conductances of the levels nf/2, nf/4, ..., nf >> nout (all of them at most
// 64 cells wide) from those of the nf-cell level above them: one block per
// sample, each level into global memory (out.cx[l], out.cy[l], per sample
// contiguous) and into shared memory, from which the next level is coarsened.
// Vertex for vertex the arithmetic of coarsen_kernel: one launch per solve
// instead of one per level.
template <typename T>
__global__ void __launch_bounds__(256) coarsen_tail_kernel(const T *__restrict__ cxf,
                                                           const T *__restrict__ cyf, int nf,
                                                           TailPtrs out, int nout) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int s = blockIdx.x;
    const long long Vf = (long long)(nf + 1) * (nf + 1);
    const T *ax = cxf + s * Vf, *ay = cyf + s * Vf;
    int nin = nf;
    for (int l = 0; l < nout; ++l) {
        const int nc = nin / 2, wc = nc + 1, Vc = wc * wc;
        T *sx = sm, *sy = sm + Vc;
        T *gx = reinterpret_cast<T *>(out.cx[l]) + (long long)s * Vc;
        T *gy = reinterpret_cast<T *>(out.cy[l]) + (long long)s * Vc;
        for (int v = threadIdx.x; v < Vc; v += blockDim.x) {
            const int J = v / wc, I = v - J * wc;
            T x, y;
            coarsen_at(ax, ay, nin, I, J, &x, &y);
            sx[v] = x;
            sy[v] = y;
            gx[v] = x;
            gy[v] = y;
        }
        __syncthreads();
        ax = sx;
        ay = sy;
        sm += 2 * Vc;
        nin = nc;
    }
}

template <typename T>
constexpr size_t coarsen_tail_smem(int nf) {
    size_t t = 0;
    for (int nc = nf / 2; nc >= 2; nc /= 2) t += 2 * (size_t)(nc + 1) * (nc + 1);
    return t * sizeof(T);
}

template <typename T>
__global__ void smooth_kernel(const T *__restrict__ cx, const T *__restrict__ cy,
                              const T *__restrict__ b, T *__restrict__ z, int n, int vpt,
                              int color, const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1;
    const T *ax = cx + s * V, *ay = cy + s * V, *bs = b + s * V;
    T *zs = z + s * V;
    FOR_VERT(V, vpt) {
        const int j = v / w, i = v - j * w;
        if (i == 0 || i == n || ((i + j) & 1) != color) continue;
        const T cw = ax[v - 1], ce = ax[v];
        const T cs = j > 0 ? ay[v - w] : T(0), cn = j < n ? ay[v] : T(0);
        T acc = bs[v] + cw * zs[v - 1] + ce * zs[v + 1];
        if (j > 0) acc += cs * zs[v - w];
        if (j < n) acc += cn * zs[v + w];
        zs[v] = smooth_div(acc, cw + ce + cs + cn);
    }
}

template <typename T>
__global__ void restrict_kernel(const T *__restrict__ cxf, const T *__restrict__ cyf,
                                const T *__restrict__ bf, const T *__restrict__ zf, int nf,
                                int vpt, T *__restrict__ bc, T *__restrict__ zc,
                                const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int nc = nf / 2;
    const long long Vf = (long long)(nf + 1) * (nf + 1), Vc = (long long)(nc + 1) * (nc + 1);
    const T *ax = cxf + s * Vf, *ay = cyf + s * Vf, *bs = bf + s * Vf, *zs = zf + s * Vf;
    const int wc = nc + 1;
    FOR_VERT(Vc, vpt) {
        const int J = v / wc, I = v - J * wc;
        bc[s * Vc + v] = (I > 0 && I < nc) ? restrict_at(ax, ay, bs, zs, nf, I, J) : T(0);
        zc[s * Vc + v] = T(0);
    }
}

template <typename T>
__global__ void prolong_kernel(const T *__restrict__ zc, int nc, T *__restrict__ zf, int vpt,
                               const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int nf = 2 * nc;
    const long long Vf = (long long)(nf + 1) * (nf + 1), Vc = (long long)(nc + 1) * (nc + 1);
    const T *c = zc + s * Vc;
    T *f = zf + s * Vf;
    const int wf = nf + 1, wc = nc + 1;
    FOR_VERT(Vf, vpt) {
        const int j = v / wf, i = v - j * wf;
        if (i == 0 || i == nf) continue;
        const int I = i >> 1, J = j >> 1;
        T val;
        if (!(i & 1) && !(j & 1)) val = c[J * wc + I];
        else if ((i & 1) && !(j & 1)) val = T(0.5) * (c[J * wc + I] + c[J * wc + I + 1]);
        else if (!(i & 1) && (j & 1)) val = T(0.5) * (c[J * wc + I] + c[(J + 1) * wc + I]);
        else
            val = T(0.25) * (c[J * wc + I] + c[J * wc + I + 1] + c[(J + 1) * wc + I] +
                             c[(J + 1) * wc + I + 1]);
        f[v] += val;
    }
}

// exact solve on the 2-cell grid: unknowns (1, j), j = 0..2, tridiagonal in j
template <typename T>
__global__ void coarsest_kernel(const T *__restrict__ cx, const T *__restrict__ cy,
                                const T *__restrict__ b, T *__restrict__ z, int count,
                                const int *__restrict__ act) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count || !act[s]) return;
    coarsest_solve(cx + s * 9, cy + s * 9, b + s * 9, z + s * 9);
}

// ---------------------------------------------------------------- Krylov pieces


template <typename T>
__global__ void dot_kernel(const T *__restrict__ a, const T *__restrict__ b, int n, int vpt,
                           double *__restrict__ part, int nblk, const int *__restrict__ act) {
    __shared__ T sh[32];
    const int s = blockIdx.y;
    if (!act[s]) return;
    const long long V = (long long)(n + 1) * (n + 1);
    T acc = T(0);
    FOR_VERT(V, vpt) acc += a[s * V + v] * b[s * V + v];
    const T tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = (double)tot;
}



// Per-sample scalar state.  ppar: the p array of the pending update (alpha, p).
// rz: two slots per sample (r.z of the iterations of even and odd parity;
// the reduction launches use the first).  rzf, alphaf: the FP32 path's folded
// r.z (float-float, two slots) and alpha.
struct Scal {
    double *rz, *pq, *rr, *rr0, *alpha, *beta, *orr, *orr0, *thr;
    float2 *rzf;
    float *alphaf;
    int *act_out, *act_in, *iters, *counter, *ppar;
};

// Fixed-order sum of one sample's nb block partials by one warp: lane-strided
// sums, then a shuffle tree; lane 0 gets the total.  Every caller (reduce_kernel
// and the blocks of the CG kernels below) adds in this order, so all of them
// obtain the same value bit for bit.
__device__ __forceinline__ double warp_sum_parts(const double *__restrict__ p, int nb, int lane) {
    double v = 0.0;
    for (int i = lane; i < nb; i += 32) v += p[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// The same fixed-order warp sum in float-float, for partials that hold FP32
// values (the block sums of the FP32 kernels): FP32 operations only, the
// result within 2^-47 of the exact sum.
template <typename P>
__device__ __forceinline__ ff warp_sum_parts_ff(const P *__restrict__ p, int nb, int lane) {
    ff v = {0.0f, 0.0f};
    for (int i = lane; i < nb; i += 32) v = ff_add_f(v, (float)p[i]);
    for (int o = 16; o > 0; o >>= 1) {
        const ff t = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, t);
    }
    return v;
}

// Where CG's scalars alpha and beta are formed (SCE_CG_FOLD): 0 = by reduction
// launches between the CG kernels; 1 = alpha inside rupdate_kernel, beta by a
// launch; 2 = both inside the CG kernels (the default).  Folded, every block
// of the consuming kernel sums the producing kernel's partials itself, in the
// fixed order of reduce_kernel; FP32 (T = float) in float-float with the
// quotient in FP32 (the kernels use alpha and beta as FP32 values), FP64 in
// FP64 (bit-identical to the launches).
enum { FOLD_NONE = 0, FOLD_ALPHA = 1, FOLD_BOTH = 2 };

// Fused CG pass of iteration k (one read of p_{k-1}): beta, p_k = z + beta
// p_{k-1}, the deferred update d += alpha_{k-1} p_{k-1} of iteration k-1
// (alpha = 0 at the start), q = A p_k and the p_k.q partials (FP32 values for
// a folded alpha on the FP32 path, else doubles).
// beta: FOLD_BOTH: from the preconditioner's r.z partials rz_part, beta =
// r.z_k / r.z_{k-1} (0 when r.z_{k-1} = 0, as at the start of an inner solve);
// r.z alternates between two slots by the parity of k: r.z_{k-1} is read from
// slot par ^ 1, block 0 stores r.z_k in slot par (no block reads that slot in
// this launch); FP32 keeps them as float-float (rzf), FP64 as doubles (rz).
// Otherwise beta[s], set by a reduction launch.  p ping-pongs: p_in holds
// p_{k-1}, p_out gets p_k; the neighbours' p_k are formed from z and p_in, so
// no block reads what another writes.  On the Dirichlet columns z = p = 0, so
// p_k stays 0 there.
template <typename T, int VPT = 0>
__global__ void pspmv_kernel(const T *__restrict__ cx, const T *__restrict__ cy,
                             const T *__restrict__ z, const T *__restrict__ p_in,
                             T *__restrict__ p_out, T *__restrict__ q, T *__restrict__ d,
                             const double *__restrict__ rz_part, int rz_nblk, Scal sc, int count,
                             int par, int fold, int n, int vpt, double *__restrict__ part,
                             int nblk, const int *__restrict__ act) {
    __shared__ T sh[32];
    __shared__ T sbeta;
    const int s = blockIdx.y;
    constexpr bool F32 = sizeof(T) == 4;
    // the per-sample scalars are loaded together with the flag (one latency)
    const T al = (F32 && fold != FOLD_NONE) ? (T)sc.alphaf[s] : (T)sc.alpha[s];
    T pre_b = T(0);
    float2 old_f = {0.0f, 0.0f};
    double old_d = 0.0;
    if (fold != FOLD_BOTH) pre_b = (T)sc.beta[s];
    else if constexpr (F32) old_f = sc.rzf[(par ^ 1) * count + s];
    else old_d = sc.rz[(par ^ 1) * count + s];
    if (!act[s]) return;
    T bt = pre_b;
    if (fold == FOLD_BOTH) {
        if (threadIdx.x < 32) {
            const double *pp = rz_part + (long long)s * rz_nblk;
            if constexpr (F32) {
                const ff v = warp_sum_parts_ff(pp, rz_nblk, threadIdx.x);
                if (threadIdx.x == 0) {
                    sbeta = old_f.x > 0.0f ? __fdiv_rn(v.hi, old_f.x) : 0.0f;
                    if (blockIdx.x == 0) sc.rzf[par * count + s] = make_float2(v.hi, v.lo);
                }
            } else {
                const double v = warp_sum_parts(pp, rz_nblk, threadIdx.x);
                if (threadIdx.x == 0) {
                    sbeta = old_d > 0.0 ? v / old_d : 0.0;
                    if (blockIdx.x == 0) sc.rz[par * count + s] = v;
                }
            }
        }
        __syncthreads();
        bt = sbeta;
    }
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1;
    const T *ax = cx + s * V, *ay = cy + s * V, *zs = z + s * V, *pi = p_in + s * V;
    T *po = p_out + s * V, *qs = q + s * V, *ds = d + s * V;
    auto pk = [&](long long u) { return zs[u] + bt * pi[u]; };
    T acc = T(0);
    FOR_VERT_C(V, VPT, vpt) {
        const int j = v / w, i = v - j * w;
        const T pold = pi[v];
        const T pc = zs[v] + bt * pold;
        po[v] = pc;
        ds[v] += al * pold;
        T val = T(0);
        if (i > 0 && i < n) {
            val = ax[v - 1] * (pc - pk(v - 1)) + ax[v] * (pc - pk(v + 1));
            if (j > 0) val += ay[v - w] * (pc - pk(v - w));
            if (j < n) val += ay[v] * (pc - pk(v + w));
            acc += pc * val;
        }
        qs[v] = val;
    }
    const T tot = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        if (F32 && fold != FOLD_NONE)
            reinterpret_cast<float *>(part)[(long long)s * nblk + blockIdx.x] = tot;
        else
            part[(long long)s * nblk + blockIdx.x] = (double)tot;
    }
}

// alpha, r -= alpha q and the r.r partials.  alpha: folded (fold != 0), every
// block sums the p.q partials of the CG pass (FP32 values on the FP32 path) in
// the same order, alpha = r.z / p.q (0 when p.q <= 0), with r.z from slot par
// of the folded state (FOLD_BOTH) or from the reduction launches' rz[s]; block
// 0 records alpha (and its FP32 copy) and the parity of the p array for the
// deferred update d += alpha p (next CG pass, or the outer update).  Not
// folded: alpha[s] from a reduction launch.  The d update itself is deferred to
// pspmv_kernel.
template <typename T, int VPT = 0>
__global__ void __launch_bounds__(256, VPT > 0 ? (sizeof(T) == 4 ? 4 : 3) : 1) rupdate_kernel(
    T *__restrict__ r, const T *__restrict__ q, const double *__restrict__ pq_part, int pq_nblk,
    Scal sc, int count, int par, int fold, int n, int vpt, double *__restrict__ part, int nblk,
    const int *__restrict__ act) {
    __shared__ T sh[32];
    __shared__ T salpha;
    const int s = blockIdx.y;
    constexpr bool F32 = sizeof(T) == 4;
    // loaded together with the flag (one latency)
    T pre_a = T(0);
    float rz_f = 0.0f;
    double rz_d = 0.0;
    if (fold == FOLD_NONE) pre_a = (T)sc.alpha[s];
    else if (fold == FOLD_BOTH) {
        if constexpr (F32) rz_f = sc.rzf[par * count + s].x;
        else rz_d = sc.rz[par * count + s];
    } else {
        if constexpr (F32) rz_f = (float)sc.rz[s];
        else rz_d = sc.rz[s];
    }
    if (!act[s]) return;
    const long long V = (long long)(n + 1) * (n + 1);
    auto alpha_of_sample = [&]() -> T {
        if (fold == FOLD_NONE) return pre_a;
        if (threadIdx.x < 32) {
            if constexpr (F32) {
                const float *pf = reinterpret_cast<const float *>(pq_part) + (long long)s * pq_nblk;
                const ff v = warp_sum_parts_ff(pf, pq_nblk, threadIdx.x);
                if (threadIdx.x == 0) {
                    const float a = v.hi > 0.0f ? __fdiv_rn(rz_f, v.hi) : 0.0f;
                    salpha = a;
                    if (blockIdx.x == 0) {
                        sc.alphaf[s] = a;
                        sc.alpha[s] = (double)a;
                        sc.ppar[s] = par;
                    }
                }
            } else {
                const double v =
                    warp_sum_parts(pq_part + (long long)s * pq_nblk, pq_nblk, threadIdx.x);
                if (threadIdx.x == 0) {
                    const double a = v > 0.0 ? rz_d / v : 0.0;
                    salpha = a;
                    if (blockIdx.x == 0) {
                        sc.alpha[s] = a;
                        sc.ppar[s] = par;
                    }
                }
            }
        }
        __syncthreads();
        return salpha;
    };
    T acc = T(0);
    if constexpr (VPT > 0) {
        // every load of the thread first (all in flight together, and while
        // alpha is formed), then the updates and stores in the same order as
        // the run-time loop
        T rv[VPT], qv[VPT];
        const long long v0 = (long long)blockIdx.x * (blockDim.x * VPT) + threadIdx.x;
#pragma unroll
        for (int e = 0; e < VPT; ++e) {
            const long long v = v0 + (long long)e * blockDim.x;
            rv[e] = v < V ? r[s * V + v] : T(0);
            qv[e] = v < V ? q[s * V + v] : T(0);
        }
        const T a = alpha_of_sample();
#pragma unroll
        for (int e = 0; e < VPT; ++e) {
            const long long v = v0 + (long long)e * blockDim.x;
            if (v < V) {
                const T t = rv[e] - a * qv[e];
                r[s * V + v] = t;
                acc += t * t;
            }
        }
    } else {
        const T a = alpha_of_sample();
        FOR_VERT_C(V, VPT, vpt) {
            const long long g = s * V + v;
            const T rv = r[g] - a * q[g];
            r[g] = rv;
            acc += rv * rv;
        }
    }
    const T tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = (double)tot;
}


enum { RED_ALPHA = 0, RED_RR = 1, RED_BETA = 2, RED_RZ0 = 3, RED_ORR = 4, RED_ORR0 = 5 };

// one warp per sample: fixed-order sum of the block partials, then the
// scalar update of `mode`.
__global__ void reduce_kernel(const double *__restrict__ part, int nblk, int count, int mode,
                              Scal sc, const int *__restrict__ act, double rtol2,
                              double in_rel2, int par) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= count) return;
    const int s = warp;
    if (act && !act[s]) return;
    const double v = warp_sum_parts(part + (long long)s * nblk, nblk, lane);
    if (lane != 0) return;
    switch (mode) {
        case RED_ALPHA:
            sc.pq[s] = v;
            sc.alpha[s] = v > 0.0 ? sc.rz[s] / v : 0.0;
            sc.ppar[s] = par;
            break;
        case RED_RR: {
            sc.rr[s] = v;
            sc.iters[s] += 1;
            const bool more = v > sc.thr[s];
            if (!more) sc.act_in[s] = 0;
            else atomicAdd(sc.counter, 1);
            break;
        }
        case RED_BETA:
            sc.beta[s] = sc.rz[s] > 0.0 ? v / sc.rz[s] : 0.0;
            sc.rz[s] = v;
            break;
        case RED_RZ0:
            sc.rz[s] = v;
            break;
        case RED_ORR:
        case RED_ORR0: {
            sc.orr[s] = v;
            if (mode == RED_ORR0) sc.orr0[s] = v;
            const bool more = v > rtol2 * sc.orr0[s] && v == v;
            sc.act_out[s] = more ? 1 : 0;
            sc.act_in[s] = sc.act_out[s];
            // inner target: relative drop in_rel2, but never below what the
            // outer tolerance needs (a quarter of it, squared: 1/16)
            sc.thr[s] = fmax(in_rel2 * v, 0.0625 * rtol2 * sc.orr0[s]);
            if (more) atomicAdd(sc.counter, 1);
            break;
        }
    }
}

// ---------------------------------------------------------------- outer refinement
// High-precision state of the refinement: FP64 path u and conductances in
// FP64 (the conductances are the hierarchy's level 0); mixed path u as
// float-float (hi, lo) pairs, conductances hi (level 0) + lo.
struct OuterD {
    double *u;
    const double *cx, *cy;
};
struct OuterF {
    float2 *u;
    const float *cx, *cy, *cxl, *cyl;
};

__device__ __forceinline__ double u_at(const OuterD &o, long long i) { return o.u[i]; }
__device__ __forceinline__ double u_at(const OuterF &o, long long i) {
    const float2 t = o.u[i];
    return (double)t.x + (double)t.y;
}
__device__ __forceinline__ double cx_at(const OuterD &o, long long i) { return o.cx[i]; }
__device__ __forceinline__ double cx_at(const OuterF &o, long long i) {
    return (double)o.cx[i] + (double)o.cxl[i];
}

// u = lifting of the Dirichlet data: 1 on x1 = 0, 0 elsewhere
// u = the bilinear prolongation of uc, the FP64 solution of the same field on
// the n/2-cell grid (the first iterate of nested iteration; the Dirichlet
// columns stay exact, means of equal values)
template <class O, int VPT = 0>
__global__ void set_u_kernel(O o, const double *__restrict__ uc, int n, int vpt) {
    const int s = blockIdx.y;
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1, nc = n / 2, wc = nc + 1;
    const double *c = uc + (long long)s * wc * wc;
    FOR_VERT_C(V, VPT, vpt) {
        const int j = v / w, i = v - j * w;
        const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
        const double u = 0.25 * ((c[j0 * wc + i0] + c[j0 * wc + i1]) +
                                 (c[j1 * wc + i0] + c[j1 * wc + i1]));
        if constexpr (std::is_same<O, OuterF>::value) {
            const ff t = ff_from_double(u);
            o.u[s * V + v] = make_float2(t.hi, t.lo);
        } else {
            o.u[s * V + v] = u;
        }
    }
}

// set_u_kernel for a float-float coarse solution (the mixed path's nested
// iteration): the mean of the one, two or four coarse values by float-float
// additions, the halving exact, so no FP64 operation per vertex.
template <int VPT = 0>
__global__ void set_u_ff_kernel(OuterF o, const float2 *__restrict__ uc, int n, int vpt,
                                unsigned long long rdm) {
    const int s = blockIdx.y;
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1, nc = n / 2, wc = nc + 1;
    const float2 *c = uc + (long long)s * wc * wc;
    auto U = [&](int jj, int ii) {
        const float2 t = c[jj * wc + ii];
        return ff{t.x, t.y};
    };
    FOR_VERT_C(V, VPT, vpt) {
        const int j = vrow(v, rdm), i = v - j * w;
        const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1;
        ff a = U(j0, i0);
        float sc = 1.0f;
        if (i1 != i0) {
            a = ff_add(a, U(j0, i1));
            sc = 0.5f;
        }
        if (j1 != j0) {
            ff b = U(j1, i0);
            if (i1 != i0) b = ff_add(b, U(j1, i1));
            a = ff_add(a, b);
            sc *= 0.5f;
        }
        o.u[s * V + v] = make_float2(a.hi * sc, a.lo * sc);
    }
}

template <class O>
__global__ void lift_kernel(O o, int n, int vpt) {
    const int s = blockIdx.y;
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1;
    FOR_VERT(V, vpt) {
        const int i = v % w;
        if constexpr (std::is_same<O, OuterF>::value) o.u[s * V + v] = make_float2(i == 0 ? 1.0f : 0.0f, 0.0f);
        else o.u[s * V + v] = i == 0 ? 1.0 : 0.0;
    }
}

// Load vector entry at a vertex of row j (F = f h^2/6 x triangles): 3 on the
// Neumann rows j = 0, n, 6 inside; Fd[0] = f h^2/2, Fd[1] = f h^2 (FP64),
// Ff the same as float-floats.
struct Load {
    double Fd[2];
    ff Ff[2];
};

// r = F - A u (unknowns; 0 on Dirichlet columns) stored as the working-precision
// right-hand side rin of the correction equation; partial sums of |r|^2.
template <typename T, class O, int VPT = 0>
__global__ void outer_residual_kernel(O o, Load F, int n, int vpt, T *__restrict__ rin,
                                      double *__restrict__ part, int nblk,
                                      const int *__restrict__ act, unsigned long long rdm) {
    __shared__ T sh[32];
    const int s = blockIdx.y;
    if (act && !act[s]) return;
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1;
    T acc = T(0);
    FOR_VERT_C(V, VPT, vpt) {
        const int j = vrow(v, rdm), i = v - j * w;
        const long long g = s * V + v;
        T rv = T(0);
        if (i > 0 && i < n) {
            const int inner = (j > 0 && j < n) ? 1 : 0;
            if constexpr (std::is_same<O, OuterF>::value) {
                const long long b0 = s * V;
                rv = resid_at_ff(inner ? F.Ff[1] : F.Ff[0], o.cx + b0, o.cxl + b0, o.cy + b0,
                                 o.cyl + b0, o.u + b0, i, j, n);
            } else {
                const double uc = o.u[g];
                double Au = o.cx[g - 1] * (uc - o.u[g - 1]) + o.cx[g] * (uc - o.u[g + 1]);
                if (j > 0) Au += o.cy[g - w] * (uc - o.u[g - w]);
                if (j < n) Au += o.cy[g] * (uc - o.u[g + w]);
                rv = (T)(F.Fd[inner] - Au);
            }
            acc += rv * rv;
        }
        rin[g] = rv;
    }
    const T tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = (double)tot;
}

// Residual of the lifting u0 (1 on x1 = 0, 0 elsewhere): A u0 is -cx(0, j) at
// the vertices (1, j) and 0 at the other unknowns, so r0 = F + [i = 1] cx(0, j).
template <typename T, class O>
__global__ void initial_residual_kernel(O o, Load F, int n, int vpt, T *__restrict__ rin,
                                        double *__restrict__ part, int nblk) {
    __shared__ T sh[32];
    const int s = blockIdx.y;
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1;
    T acc = T(0);
    FOR_VERT(V, vpt) {
        const int j = v / w, i = v - j * w;
        const long long g = s * V + v;
        T rv = T(0);
        if (i > 0 && i < n) {
            const int inner = (j > 0 && j < n) ? 1 : 0;
            if constexpr (std::is_same<O, OuterF>::value) {
                ff r = F.Ff[inner];
                if (i == 1) r = ff_add(r, ff{o.cx[g - 1], o.cxl[g - 1]});
                rv = r.hi;
            } else {
                double r = F.Fd[inner];
                if (i == 1) r += o.cx[g - 1];
                rv = (T)r;
            }
            acc += rv * rv;
        }
        rin[g] = rv;
    }
    const T tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(long long)s * nblk + blockIdx.x] = (double)tot;
}

// u += d + alpha p: the inner solve's correction with its last deferred CG
// update (alpha and the p array ppar of the sample's last iteration; alpha = 0
// when none is pending).  float-float + float on the mixed path.
template <typename T, class O, int VPT = 0>
__global__ void outer_update_kernel(O o, const T *__restrict__ d, const T *__restrict__ p0,
                                    const T *__restrict__ p1, const double *__restrict__ alpha,
                                    const int *__restrict__ ppar, int n, int vpt,
                                    const int *__restrict__ act) {
    const int s = blockIdx.y;
    if (!act[s]) return;
    const long long V = (long long)(n + 1) * (n + 1);
    const T a = (T)alpha[s];
    const T *p = ppar[s] ? p1 : p0;
    if constexpr (VPT > 0 && std::is_same<O, OuterF>::value) {
        // every load of the thread first, then the updates
        float2 uv[VPT];
        T dv[VPT];
        const long long v0 = (long long)blockIdx.x * (blockDim.x * VPT) + threadIdx.x;
#pragma unroll
        for (int e = 0; e < VPT; ++e) {
            const long long v = v0 + (long long)e * blockDim.x;
            const long long g = s * V + (v < V ? v : 0);
            uv[e] = o.u[g];
            dv[e] = d[g] + a * p[g];
        }
#pragma unroll
        for (int e = 0; e < VPT; ++e) {
            const long long v = v0 + (long long)e * blockDim.x;
            if (v < V) {
                const ff r = ff_add_f(ff{uv[e].x, uv[e].y}, (float)dv[e]);
                o.u[s * V + v] = make_float2(r.hi, r.lo);
            }
        }
        return;
    }
    FOR_VERT_C(V, VPT, vpt) {
        const long long g = s * V + v;
        const T dv = d[g] + a * p[g];
        if constexpr (std::is_same<O, OuterF>::value) {
            const float2 t = o.u[g];
            const ff r = ff_add_f(ff{t.x, t.y}, (float)dv);
            o.u[g] = make_float2(r.hi, r.lo);
        } else {
            o.u[g] += (double)dv;
        }
    }
}

template <class O>
__global__ void u_to_double_kernel(O o, int n, int vpt, double *__restrict__ out) {
    const int s = blockIdx.y;
    const long long V = (long long)(n + 1) * (n + 1);
    FOR_VERT(V, vpt) out[s * V + v] = u_at(o, s * V + v);
}

// QoI partials: outflow (vertices i = n-1; bit 0 of qmask) and the P1 mass
// norm (cells; bit 2).
template <class O>
__global__ void qoi_partial_kernel(O o, int n, int vpt, double *__restrict__ part_out,
                                   double *__restrict__ part_l2, int nblk, int qmask) {
    __shared__ double sh[32];
    const int s = blockIdx.y;
    const long long V = (long long)(n + 1) * (n + 1);
    const int w = n + 1;
    const long long g0 = s * V;
    const bool want_out = qmask & 1, want_l2 = qmask & 4;
    double qo = 0.0, l2 = 0.0;
    FOR_VERT(V, vpt) {
        const int j = v / w, i = v - j * w;
        if (want_out && i == n - 1) qo += cx_at(o, g0 + v) * u_at(o, g0 + v);
        if (want_l2 && i < n && j < n) {
            const double a = u_at(o, g0 + v), b = u_at(o, g0 + v + 1);
            const double c = u_at(o, g0 + v + w + 1), d = u_at(o, g0 + v + w);
            const double s1 = a + b + c, s2 = a + d + c;
            l2 += s1 * s1 + a * a + b * b + c * c + s2 * s2 + a * a + d * d + c * c;
        }
    }
    double t = block_sum(qo, sh);
    if (threadIdx.x == 0) part_out[(long long)s * nblk + blockIdx.x] = t;
    t = block_sum(l2, sh);
    if (threadIdx.x == 0) part_l2[(long long)s * nblk + blockIdx.x] = t;
}

// QoIs per sample (those of qmask; the others are written as 0), status,
// iteration counts.  part_out / part_l2 may be NULL when qmask has neither.
template <class O>
__global__ void qoi_final_kernel(const double *__restrict__ part_out,
                                 const double *__restrict__ part_l2, int nblk, int count,
                                 O o, int n, double f,
                                 const Scal sc, double rtol2, double *__restrict__ qoi,
                                 int *__restrict__ iters_out, int *__restrict__ status_out,
                                 int *__restrict__ nfail, int qmask) {
    // nfail[0]: samples that failed; nfail[1], nfail[2]: the largest and the
    // total iteration count (integer atomics: order-independent)
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= count) return;
    const int s = warp;
    double a = 0.0, b = 0.0;
    if (part_out) {
        for (int i = lane; i < nblk; i += 32) {
            a += part_out[(long long)s * nblk + i];
            b += part_l2[(long long)s * nblk + i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane != 0) return;
    const double h = 1.0 / (double)n;
    const double q_out = a + f * h * 0.5;
    const double q_l2 = sqrt(b * h * h / 24.0);
    // point value at (7/15, 7/15): cell (ca, cb), local (xi, eta)
    const double xs = 7.0 / 15.0 * (double)n, ys = 7.0 / 15.0 * (double)n;
    const int ca = min((int)floor(xs), n - 1), cb = min((int)floor(ys), n - 1);
    const double xi = xs - ca, et = ys - cb;
    const long long V = (long long)(n + 1) * (n + 1);
    const long long g0 = s * V;
    const int w = n + 1;
    const double uab = u_at(o, g0 + cb * w + ca), ua1b = u_at(o, g0 + cb * w + ca + 1);
    const double uab1 = u_at(o, g0 + (cb + 1) * w + ca);
    const double ua1b1 = u_at(o, g0 + (cb + 1) * w + ca + 1);
    double q_pt;
    if (xi >= et) q_pt = uab + xi * (ua1b - uab) + et * (ua1b1 - ua1b);   // T1
    else q_pt = uab + et * (uab1 - uab) + xi * (ua1b1 - uab1);             // T2
    qoi[3 * s + 0] = (qmask & 1) ? q_out : 0.0;
    qoi[3 * s + 1] = (qmask & 2) ? q_pt : 0.0;
    qoi[3 * s + 2] = (qmask & 4) ? q_l2 : 0.0;
    int st = 0;
    if (!(fabs(qoi[3 * s]) < 1e300 && fabs(qoi[3 * s + 1]) < 1e300 && fabs(qoi[3 * s + 2]) < 1e300))
        st = CE_ERR_NONFINITE;
    else if (!(sc.orr[s] <= rtol2 * sc.orr0[s])) st = CE_ERR_NOT_CONVERGED;
    if (status_out) status_out[s] = st;
    const int its = sc.iters[s];
    if (iters_out) iters_out[s] = its;
    if (st != 0) atomicAdd(nfail, 1);
    atomicMax(nfail + 1, its);
    atomicAdd(nfail + 2, its);
}

// ---------------------------------------------------------------- host driver
template <typename T>
struct Solver {
    int count = 0, nlev = 0;
    int n[MAXLEV];
    Launch ln[MAXLEV];
    T *cx[MAXLEV], *cy[MAXLEV], *b[MAXLEV], *z[MAXLEV];
    T *zpre[MAXLEV] = {};   // pre-smoothed z of the tiled levels (fused cycle)
    T *d = nullptr, *p = nullptr, *q = nullptr;
    T *p2 = nullptr;   // second p array (p ping-pongs between p and p2)
    int par = 0;       // the array the next fused pass writes: 0 = p, 1 = p2
    double *u64 = nullptr;                  // FP64 path: u
    float2 *uff = nullptr;                  // mixed path: u as float-float pairs
    float *cxl = nullptr, *cyl = nullptr;   // mixed path: lo parts of the conductances
    double *part = nullptr, *part2 = nullptr;
    Scal sc{};
    int *misc = nullptr;   // [0] counter, [1] nfail, [2] max iters, [3] total iters
    std::vector<void *> owned;
    cudaStream_t st = nullptr;
    cudaGraphExec_t graph = nullptr;   // four captured CG iterations, replayed

    template <typename U> int alloc(U **ptr, size_t cnt) {
        int rc = sce_alloc_t(ptr, cnt, st);
        if (rc == CE_OK) owned.push_back((void *)*ptr);
        return rc;
    }
    ~Solver() {
        if (graph) cudaGraphExecDestroy(graph);
        for (void *ptr : owned) sce_free(ptr, st);
    }

    dim3 grid(int L) const { return dim3(ln[L].nblk, count); }

    double vb(int L, double per_vertex_T, double extra_bytes = 0.0) const {
        return (double)count * (double)ln[L].V * (per_vertex_T * sizeof(T) + extra_bytes);
    }

    int smooth(int L, int color) {
        SceProf pr(KP_SMOOTH, st, vb(L, 3.5));
        smooth_kernel<T><<<grid(L), ln[L].tpb, 0, st>>>(cx[L], cy[L], b[L], z[L], n[L], ln[L].vpt,
                                                        color, sc.act_in);
        return CE_OK;
    }

    void vcycle(int L) {
        if (n[L] == 2) {
            SceProf pr(KP_COARSEST, st, vb(L, 4.0));
            coarsest_kernel<T><<<(count + 127) / 128, 128, 0, st>>>(cx[L], cy[L], b[L], z[L], count,
                                                                    sc.act_in);
            return;
        }
        for (int k = 0; k < lnu(L); ++k) {
            smooth(L, 0);
            smooth(L, 1);
        }
        {
            SceProf pr(KP_RESTRICT, st, vb(L, 4.0) + vb(L + 1, 2.0));
            restrict_kernel<T><<<grid(L + 1), ln[L + 1].tpb, 0, st>>>(
                cx[L], cy[L], b[L], z[L], n[L], ln[L + 1].vpt, b[L + 1], z[L + 1], sc.act_in);
        }
        vcycle(L + 1);
        {
            SceProf pr(KP_PROLONG, st, vb(L, 2.0) + vb(L + 1, 1.0));
            prolong_kernel<T><<<grid(L), ln[L].tpb, 0, st>>>(z[L + 1], n[L + 1], z[L], ln[L].vpt,
                                                             sc.act_in);
        }
        for (int k = 0; k < lnu(L); ++k) {
            smooth(L, 1);
            smooth(L, 0);
        }
    }

    // ---- fused cycle: tiled down/up kernels above the tail, one block per
    // sample for the levels n <= TAIL_N
    bool fused = true;
    int Lt = 0;                 // first level of the tail
    int tiles_x[MAXLEV], tiles_n[MAXLEV], sh[MAXLEV];
    int nu[MAXLEV];             // sweeps per side of each tiled level
    int nu_c = 0;               // sweeps per side of the coarse levels (FP32)
    int v64_nut = 0, v64_nus = 0;
    // sweeps per side on level L, the same rule on every path of the cycle
    // (tiles, fused n = 64 cycle, one-block tail, level-by-level kernels)
    int lnu(int L) const {
        return (n[0] >= 2 * V64_N && L > 0 && L < nlev && n[L] <= MG_NU_COARSE_MAX)
                   ? nu_c
                   : mg_nu<T>();
    }

    // FP32: an n = 64 level and everything below it run as one fused kernel
    // per sample (mg_v64_kernel; SCE_V64=0 keeps the tiled kernels for it)
    bool v64 = false;

    void plan_fused() {
        int tail_n = TAIL_N;
        if constexpr (sizeof(T) == 4) {
            const char *e = getenv("SCE_V64");
            if (!(e && atoi(e) == 0) && TAIL_N < V64_N) tail_n = V64_N;
        }
        Lt = 0;
        while (n[Lt] > tail_n) ++Lt;
        v64 = sizeof(T) == 4 && tail_n == V64_N && n[Lt] == V64_N;
        nu_c = sizeof(T) == 4 ? mg_nu_coarse() : mg_nu<T>();
        v64_nut = lnu(Lt);
        v64_nus = lnu(Lt + 1);
        for (int L = 0; L < Lt; ++L) {
            const int nc1 = n[L] / 2 + 1;
            nu[L] = lnu(L);
            sh[L] = tile_height_for((int)sizeof(T), n[L]);
            // three sweeps: windows of 48 rows (CH = SH / 2 - 7), or 64 where the
            // table or SCE_TILE_SH3=64 asks for them
            if (nu[L] == 3) {
                const char *e3 = getenv("SCE_TILE_SH3");
                sh[L] = (sh[L] == 64 || (e3 && atoi(e3) == 64)) ? 64 : 48;
            }
            const int ch = nu[L] == 3 ? MGGeom<T, 3>::ch(sh[L]) : MGGeom<T>::ch(sh[L]);
            const int cw = nu[L] == 3 ? MGGeom<T, 3>::CW : MGGeom<T>::CW;
            tiles_x[L] = (nc1 + cw - 1) / cw;
            tiles_n[L] = tiles_x[L] * ((nc1 + ch - 1) / ch);
        }
    }

    // levels and launch plan of an n0-cell hierarchy of `cnt` samples (no allocation)
    void init_plan(int n0, int cnt) {
        count = cnt;
        int lv = 0;
        for (int nn = n0; nn >= 2; nn /= 2) {
            n[lv] = nn;
            ln[lv] = launch_for(nn);
            ++lv;
        }
        nlev = lv;
        const char *e = getenv("SCE_MG_FUSED");
        fused = !(e && atoi(e) == 0);
        plan_fused();
    }

    // what a cached solver must match to be reused: samples, grid and plan
    std::vector<int> signature() const {
        std::vector<int> sg{count, n[0], fused ? 1 : 0, Lt, v64 ? 1 : 0, nu_c};
        for (int L = 0; L < Lt; ++L) sg.push_back(sh[L]);
        return sg;
    }

    int alloc_all() {
        for (int L = 0; L < nlev; ++L) {
            const size_t cnt = (size_t)count * ln[L].V;
            SCE_TRY(alloc(&cx[L], cnt));
            SCE_TRY(alloc(&cy[L], cnt));
            SCE_TRY(alloc(&b[L], cnt));
            SCE_TRY(alloc(&z[L], cnt));
        }
        const size_t c0 = (size_t)count * ln[0].V;
        SCE_TRY(alloc(&d, c0));
        SCE_TRY(alloc(&p, c0));
        SCE_TRY(alloc(&p2, c0));
        SCE_TRY(alloc(&q, c0));
        if constexpr (sizeof(T) == 4) {
            SCE_TRY(alloc(&uff, c0));
            SCE_TRY(alloc(&cxl, c0));
            SCE_TRY(alloc(&cyl, c0));
        } else {
            SCE_TRY(alloc(&u64, c0));
        }
        if (fused)
            for (int L = 0; L < Lt; ++L) SCE_TRY(alloc(&zpre[L], (size_t)count * ln[L].V));
        const int nblk_part = std::max(ln[0].nblk, rz_blocks());
        SCE_TRY(alloc(&part, (size_t)count * nblk_part));
        SCE_TRY(alloc(&part2, (size_t)count * nblk_part));
        double *scal = nullptr;
        SCE_TRY(alloc(&scal, (size_t)count * 10));
        sc.rz = scal;   // two slots
        sc.pq = scal + 2 * count;
        sc.rr = scal + 3 * count;
        sc.rr0 = scal + 4 * count;
        sc.alpha = scal + 5 * count;
        sc.beta = scal + 6 * count;
        sc.orr = scal + 7 * count;
        sc.orr0 = scal + 8 * count;
        sc.thr = scal + 9 * count;
        SCE_TRY(alloc(&sc.rzf, (size_t)count * 2));
        SCE_TRY(alloc(&sc.alphaf, (size_t)count));
        int *ints = nullptr;
        SCE_TRY(alloc(&ints, (size_t)count * 4 + 4));
        sc.act_out = ints;
        sc.act_in = ints + count;
        sc.iters = ints + 2 * count;
        sc.ppar = ints + 3 * count;
        misc = ints + 4 * count;
        sc.counter = misc;
        return CE_OK;
    }

    // launches of the tiled kernels of window height SH and NU sweeps per side
    unsigned tile_attr_mask = 0;
    template <int SH, int NU>
    void tile_down(int L) {
        constexpr size_t smem = mg_tile_smem_bytes<T, SH>();
        constexpr unsigned bit = 1u << (SH / 8 + 9 * (NU - 1));
        if (!(tile_attr_mask & bit)) {   // outside any capture (the first cycle is not captured)
            sce_raise_smem_limit((const void *)mg_down_kernel<T, SH, NU>, smem);
            sce_raise_smem_limit((const void *)mg_up_kernel<T, SH, NU>, smem);
            tile_attr_mask |= bit;
        }
        SceProf pr(NU == 3 ? KP_MG_DOWN3 : KP_MG_DOWN, st, vb(L, 4.0) + vb(L + 1, 1.0));
        mg_down_kernel<T, SH, NU><<<dim3(tiles_n[L], count), MGTile<SH>::THREADS, smem, st>>>(
            cx[L], cy[L], b[L], zpre[L], n[L], b[L + 1], tiles_x[L], sc.act_in);
    }
    template <int SH, int NU>
    void tile_up(int L, bool want_rz) {
        constexpr size_t smem = mg_tile_smem_bytes<T, SH>();
        SceProf pr(NU == 3 ? KP_MG_UP3 : KP_MG_UP, st, vb(L, 5.0) + vb(L + 1, 1.0));
        mg_up_kernel<T, SH, NU><<<dim3(tiles_n[L], count), MGTile<SH>::THREADS, smem, st>>>(
            cx[L], cy[L], b[L], zpre[L], z[L], n[L], z[L + 1], tiles_x[L], sc.act_in,
            (want_rz && L == 0) ? part : nullptr, tiles_n[0]);
    }
    // by the level's window height and sweep count (three sweeps: FP32, 48 or
    // 64 rows)
    template <int NU>
    void tile_pass(int L, bool up, bool want_rz) {
        auto go = [&](auto shc) {
            constexpr int SH = decltype(shc)::value;
            if (up) tile_up<SH, NU>(L, want_rz);
            else tile_down<SH, NU>(L);
        };
        if constexpr (NU == 3) {
            if (sh[L] == 64) go(std::integral_constant<int, 64>{});
            else go(std::integral_constant<int, 48>{});
        } else {
            switch (sh[L]) {
                case 16: go(std::integral_constant<int, 16>{}); break;
                case 24: go(std::integral_constant<int, 24>{}); break;
                case 48: go(std::integral_constant<int, 48>{}); break;
                case 64: go(std::integral_constant<int, 64>{}); break;
                default: go(std::integral_constant<int, 32>{}); break;
            }
        }
    }
    void tile_level(int L, bool up, bool want_rz) {
        if constexpr (sizeof(T) == 4) {
            if (nu[L] == 3) {
                tile_pass<3>(L, up, want_rz);
                return;
            }
        }
        tile_pass<mg_nu<T>()>(L, up, want_rz);
    }

    // partial-sum slots per sample written by vcycle_fused(want_rz = true)
    int rz_blocks() const { return Lt == 0 ? 1 : tiles_n[0]; }

    bool tail_attr_set = false;
    bool ctail_attr_set = false;   // shared-memory limit of coarsen_tail_kernel raised
    template <int NTN, int NTHR>
    void tail_launch(bool want_rz) {
        TailPtrs tp{};
        for (int i = 0; Lt + i < nlev && i < 8; ++i) {
            tp.cx[i] = cx[Lt + i];
            tp.cy[i] = cy[Lt + i];
        }
        constexpr size_t smem = tail_smem_bytes<T, NTN>();
        if (!tail_attr_set) {   // set outside any stream capture (the first cycle is not captured)
            sce_raise_smem_limit((const void *)mg_tail_kernel<T, NTN, NTHR>, smem);
            tail_attr_set = true;
        }
        SceProf pr(KP_MG_TAIL, st, (double)count * (smem + 2 * sizeof(T) * ln[Lt].V));
        mg_tail_kernel<T, NTN, NTHR><<<count, NTHR, smem, st>>>(tp, b[Lt], z[Lt], sc.act_in,
                                                                want_rz ? part : nullptr,
                                                                lnu(Lt), lnu(Lt + 1));
    }

    unsigned v64_attr_mask = 0;
    template <int NUT, int NUS, bool PAD>
    void v64_go(const TailPtrs &tp, double *pr_rz) {
        constexpr size_t smem = v64_smem_bytes<T, PAD>();
        constexpr unsigned bit = 1u << (NUT * 4 + NUS + (PAD ? 16 : 0));
        if (!(v64_attr_mask & bit)) {   // outside any stream capture (the first cycle is not captured)
            sce_raise_smem_limit((const void *)mg_v64_kernel<T, 0, NUT, NUS, PAD>, smem);
            v64_attr_mask |= bit;
        }
        mg_v64_kernel<T, 0, NUT, NUS, PAD><<<count, V64_THREADS, smem, st>>>(
            cx[Lt], cy[Lt], b[Lt], z[Lt], tp, sc.act_in, pr_rz);
    }
    template <int NUT, int NUS>
    void v64_go(const TailPtrs &tp, double *pr_rz) {
        if (sce_smem_pad()) v64_go<NUT, NUS, true>(tp, pr_rz);
        else v64_go<NUT, NUS, false>(tp, pr_rz);
    }
    void v64_launch(bool want_rz) {
        if constexpr (sizeof(T) == 4) {
            TailPtrs tp{};
            for (int i = 0; Lt + 1 + i < nlev && i < 8; ++i) {
                tp.cx[i] = cx[Lt + 1 + i];
                tp.cy[i] = cy[Lt + 1 + i];
            }
            // b, cx, cy in, z out on the level; the conductances of the levels below in
            double tail_v = 0.0;
            for (int L = Lt + 1; L < nlev; ++L) tail_v += (double)ln[L].V;
            SceProf pr(KP_MG_V64, st, vb(Lt, 4.0) + (double)count * tail_v * 2.0 * sizeof(T));
            double *pr_rz = want_rz ? part : nullptr;
            // three sweeps on the n = 64 level and below when it is a coarse
            // level of a wider grid, else the default
            if (v64_nut == 3 && v64_nus == 3) v64_go<3, 3>(tp, pr_rz);
            else v64_go<mg_nu<T>(), mg_nu<T>()>(tp, pr_rz);
        }
    }

    // z[0] = M^{-1} b[0]; with want_rz the partial sums of b[0] . z[0] go to part
    void vcycle_fused(bool want_rz) {
        for (int L = 0; L < Lt; ++L) tile_level(L, false, false);
        const bool rz_tail = want_rz && Lt == 0;
        if (v64) v64_launch(rz_tail);
        else switch (n[Lt]) {
            case 64: tail_launch<64, 512>(rz_tail); break;
            case 32: tail_launch<32, 256>(rz_tail); break;
            case 16: tail_launch<16, 128>(rz_tail); break;
            case 8: tail_launch<8, 64>(rz_tail); break;
            default: tail_launch<4, 32>(rz_tail); break;
        }
        for (int L = Lt - 1; L >= 0; --L) tile_level(L, true, want_rz);
    }

    void reduce(int mode, const int *act, double rtol2 = 0.0, double in_rel2 = 0.0,
                int nblk = -1, int rpar = 0, const double *src = nullptr) {
        const int threads = 256;
        const int blocks = (count * 32 + threads - 1) / threads;
        if (nblk < 0) nblk = ln[0].nblk;
        SceProf pr(KP_REDUCE, st, (double)count * nblk * 8.0);
        reduce_kernel<<<blocks, threads, 0, st>>>(src ? src : part, nblk, count, mode, sc, act,
                                                  rtol2, in_rel2, rpar);
    }

    int read_counter(int *host) {
        SCE_CUDA(cudaMemcpyAsync(host, sc.counter, sizeof(int), cudaMemcpyDeviceToHost, st));
        SCE_CUDA(cudaStreamSynchronize(st));
        return CE_OK;
    }
};

// ---- idle solvers of earlier calls, with their captured CG iterations
// (SCE_GRAPHS=1).  A solve takes an idle solver of the same plan (samples,
// grid, window heights) or builds one; a successful solve puts it back, a
// failed one destroys it.  At most kPoolMax idle solvers are kept (the least
// recently used is freed); darcy_solver_cache_clear frees them all.
constexpr int kPoolMax = 16;

static // Where CG's alpha and beta are formed: SCE_CG_FOLD = 0 (reduction launches),
// 1 (alpha folded into the r update) or 2 (both folded; the default).
int cg_fold_mode() {
    const char *e = getenv("SCE_CG_FOLD");
    if (!e) return FOLD_BOTH;
    const int v = atoi(e);
    return (v == FOLD_NONE || v == FOLD_ALPHA) ? v : FOLD_BOTH;
}

bool solver_graphs_on(cudaStream_t st) {
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread || sce_prof_on())
        return false;
    const char *e = getenv("SCE_GRAPHS");
    if (!(e && atoi(e) != 0)) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

template <typename T>
struct SolverPool {
    std::mutex mu;
    std::vector<std::pair<int, Solver<T> *>> idle;   // (device, solver), most recent last

    Solver<T> *take(const std::vector<int> &sig) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = idle.size(); i-- > 0;) {
            if (idle[i].first == dev && idle[i].second->signature() == sig) {
                Solver<T> *s = idle[i].second;
                idle.erase(idle.begin() + (long)i);
                return s;
            }
        }
        return nullptr;
    }
    void give(Solver<T> *s, cudaStream_t st) {
        int dev = 0;
        cudaGetDevice(&dev);
        std::vector<Solver<T> *> victims;
        {
            std::lock_guard<std::mutex> lk(mu);
            idle.emplace_back(dev, s);
            // at most kPoolMax idle solvers of this device: the least recently
            // used of them are freed (on this device, stream-ordered on st)
            int mine = 0;
            for (auto &pr : idle) mine += pr.first == dev;
            for (size_t i = 0; i < idle.size() && mine > kPoolMax;) {
                if (idle[i].first == dev) {
                    victims.push_back(idle[i].second);
                    idle.erase(idle.begin() + (long)i);
                    --mine;
                } else {
                    ++i;
                }
            }
        }
        for (Solver<T> *v : victims) {   // their last solve has finished (solves synchronise)
            v->st = st;
            delete v;
        }
    }
    int clear(cudaStream_t st) {
        std::vector<std::pair<int, Solver<T> *>> all;
        {
            std::lock_guard<std::mutex> lk(mu);
            all.swap(idle);
        }
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess) return CE_ERR_CUDA;
        for (auto &pr : all) {
            cudaSetDevice(pr.first);
            pr.second->st = pr.first == cur ? st : nullptr;
            delete pr.second;
        }
        cudaSetDevice(cur);
        return CE_OK;
    }
};

template <typename T>
SolverPool<T> &solver_pool() {
    static SolverPool<T> pool;
    return pool;
}

// Owns the solver of one solve: back to the pool on success (cached mode),
// destroyed otherwise.
template <typename T>
struct SolverLease {
    bool cached;
    cudaStream_t st;
    Solver<T> *s = nullptr;
    bool ok = false;
    SolverLease(bool c, cudaStream_t stream) : cached(c), st(stream) {}
    ~SolverLease() {
        if (!s) return;
        if (cached && ok) solver_pool<T>().give(s, st);
        else delete s;
    }
};

template <typename T, typename Tk>
static int darcy_solve_t(const darcy_problem *p, const Tk *k, int count, double *qoi, int *iters,
                         int *status, double *u_out, cudaStream_t st, int *max_iters_out,
                         int *n_failed_out, int qmask, const double *u_init, bool u_ff) {
    // the solver's buffers, and with cached graphs the captured iterations,
    // come from the pool of idle solvers of the same plan when there is one
    const bool cached = solver_graphs_on(st);
    SolverLease<T> lease(cached, st);
    {
        auto fresh = std::make_unique<Solver<T>>();
        fresh->st = st;
        fresh->init_plan(p->n, count);
        Solver<T> *hit = cached ? solver_pool<T>().take(fresh->signature()) : nullptr;
        if (hit) {
            lease.s = hit;
        } else {
            SCE_TRY(fresh->alloc_all());
            lease.s = fresh.release();
        }
    }
    Solver<T> &S = *lease.s;
    S.st = st;
    const int n0 = p->n;
    const long long V0 = S.ln[0].V;
    const size_t c0 = (size_t)count * V0;
    constexpr bool mixed = sizeof(T) == 4;
    using O = std::conditional_t<mixed, OuterF, OuterD>;
    O o{};
    if constexpr (mixed) o = OuterF{S.uff, S.cx[0], S.cy[0], S.cxl, S.cyl};
    else o = OuterD{S.u64, S.cx[0], S.cy[0]};
    Load F{};
    {
        const double h2_6 = p->f / (6.0 * (double)n0 * (double)n0);
        F.Fd[0] = h2_6 * 3.0;   // 3 triangles at a vertex of the rows j = 0, n
        F.Fd[1] = h2_6 * 6.0;
        for (int r = 0; r < 2; ++r) {
            F.Ff[r].hi = (float)F.Fd[r];
            F.Ff[r].lo = (float)(F.Fd[r] - (double)F.Ff[r].hi);
        }
    }
    // both p arrays start finite (the first fused pass multiplies p_in by 0)
    SCE_CUDA(cudaMemsetAsync(S.p, 0, c0 * sizeof(T), st));
    SCE_CUDA(cudaMemsetAsync(S.p2, 0, c0 * sizeof(T), st));
    SCE_CUDA(cudaMemsetAsync(S.sc.act_out, 0, ((size_t)count * 4 + 4) * sizeof(int), st));

    const Launch &l0 = S.ln[0];
    const dim3 g0 = S.grid(0);
    // operator and hierarchy
    {
        SceProf pr(KP_COND, st, S.vb(0, 2.0, sizeof(Tk) + (mixed ? 8.0 : 0.0)));
        if (l0.vpt == 8)
            cond_kernel<Tk, T, 8><<<g0, l0.tpb, 0, st>>>(k, n0, 8, S.cx[0], S.cy[0], S.cxl, S.cyl,
                                                         row_magic(n0 + 1));
        else
            cond_kernel<Tk, T><<<g0, l0.tpb, 0, st>>>(k, n0, l0.vpt, S.cx[0], S.cy[0], S.cxl,
                                                      S.cyl, row_magic(n0 + 1));
    }
    SCE_CUDA(cudaGetLastError());
    // levels wider than 64 cells one launch each, then every narrower level
    // in one launch
    int Lc = 1;
    for (; Lc < S.nlev && S.n[Lc] > 64; ++Lc) {
        const int L = Lc;
        SceProf pr(KP_COARSEN, st, S.vb(L - 1, 2.0) + S.vb(L, 2.0));
        if (S.ln[L].vpt == 8)
            coarsen_kernel<T, 8><<<S.grid(L), S.ln[L].tpb, 0, st>>>(
                S.cx[L - 1], S.cy[L - 1], S.n[L - 1], 8, S.cx[L], S.cy[L], row_magic(S.n[L] + 1));
        else
            coarsen_kernel<T><<<S.grid(L), S.ln[L].tpb, 0, st>>>(
                S.cx[L - 1], S.cy[L - 1], S.n[L - 1], S.ln[L].vpt, S.cx[L], S.cy[L],
                row_magic(S.n[L] + 1));
    }
    if (Lc < S.nlev) {
        const int nout = S.nlev - Lc;
        double bytes = S.vb(Lc - 1, 2.0);
        TailPtrs outp{};
        for (int l = 0; l < nout; ++l) {
            outp.cx[l] = S.cx[Lc + l];
            outp.cy[l] = S.cy[Lc + l];
            bytes += S.vb(Lc + l, 2.0);
        }
        const size_t smem = coarsen_tail_smem<T>(S.n[Lc - 1]);
        if (!S.ctail_attr_set) {   // the largest tail (from a 128-cell level)
            SCE_TRY(sce_raise_smem_limit((const void *)coarsen_tail_kernel<T>,
                                         coarsen_tail_smem<T>(128)));
            S.ctail_attr_set = true;
        }
        SceProf pr(KP_COARSEN_TAIL, st, bytes);
        coarsen_tail_kernel<T><<<count, 256, smem, st>>>(S.cx[Lc - 1], S.cy[Lc - 1],
                                                         S.n[Lc - 1], outp, nout);
    }
    SCE_CUDA(cudaGetLastError());
    // u = the lifting of the Dirichlet data, unless a first iterate is given
    // (set_u_kernel below then writes every vertex of u)
    if (!u_init) {
        SceProf pr(KP_OUTER_UPD, st, S.vb(0, 0.0, 8.0));
        lift_kernel<<<g0, l0.tpb, 0, st>>>(o, n0, l0.vpt);
    }

    const double rtol2 = p->rtol * p->rtol;
    const double in_rel = sizeof(T) == 4 ? sce_inner_rel_f32() : 0.0;
    const double in_rel2 = in_rel * in_rel;
    const int maxit = p->maxit > 0 ? p->maxit : 1000;
    const int inner_max = sizeof(T) == 4 ? 40 : maxit;
    // iterations between host reads of the active-sample count (the per-sample
    // flags stop converged samples in between, but their blocks still launch):
    // SCE_CHECK_EVERY, default 2 (V(2,2) inner solves take ~5 iterations, so
    // checking every 4 launched ~8)
    const int check_every = [] {
        const char *e = getenv("SCE_CHECK_EVERY");
        const int v = e ? atoi(e) : 2;
        return (v >= 1 && v <= 8) ? v : 2;
    }();

    // initial residual (of the lifting, in closed form)
    {
        SceProf pr(KP_OUTER_RES, st, S.vb(0, 1.0));
        initial_residual_kernel<T><<<g0, l0.tpb, 0, st>>>(o, F, n0, l0.vpt, S.b[0], S.part,
                                                          l0.nblk);
    }
    SCE_CUDA(cudaMemsetAsync(S.sc.counter, 0, sizeof(int), st));
    S.reduce(RED_ORR0, nullptr, rtol2, in_rel2);
    SCE_CUDA(cudaGetLastError());
    // a given first iterate: the stopping rule stays relative to the lifting's
    // residual (orr0 above); refinement starts from u_init's residual
    if (u_init) {
        {
            // reads the coarse solution (8 B per coarse vertex), writes u (8 B)
            SceProf pr(KP_OUTER_UPD, st, S.vb(0, 0.0, 10.0));
            if constexpr (mixed) {
                if (u_ff) {
                    const float2 *uf = reinterpret_cast<const float2 *>(u_init);
                    if (l0.vpt == 8)
                        set_u_ff_kernel<8><<<g0, l0.tpb, 0, st>>>(o, uf, n0, 8, row_magic(n0 + 1));
                    else
                        set_u_ff_kernel<><<<g0, l0.tpb, 0, st>>>(o, uf, n0, l0.vpt,
                                                                 row_magic(n0 + 1));
                }
            }
            if (!(mixed && u_ff)) {
                if (l0.vpt == 8) set_u_kernel<O, 8><<<g0, l0.tpb, 0, st>>>(o, u_init, n0, 8);
                else set_u_kernel<O><<<g0, l0.tpb, 0, st>>>(o, u_init, n0, l0.vpt);
            }
        }
        {
            SceProf pr(KP_OUTER_RES, st, S.vb(0, 1.0, 24.0));
            if (l0.vpt == 8)
                outer_residual_kernel<T, O, 8><<<g0, l0.tpb, 0, st>>>(
                    o, F, n0, 8, S.b[0], S.part, l0.nblk, S.sc.act_out, row_magic(n0 + 1));
            else
                outer_residual_kernel<T, O><<<g0, l0.tpb, 0, st>>>(
                    o, F, n0, l0.vpt, S.b[0], S.part, l0.nblk, S.sc.act_out,
                    row_magic(n0 + 1));
        }
        SCE_CUDA(cudaMemsetAsync(S.sc.counter, 0, sizeof(int), st));
        S.reduce(RED_ORR, S.sc.act_out, rtol2, in_rel2);
        SCE_CUDA(cudaGetLastError());
    }
    int n_act = 0;
    // launch profiler (when on): the CG loop's kernels are charged for all
    // samples at launch; the passes that ran are counted at the end
    const SceProfMark prof_mark = sce_prof_on() ? sce_prof_mark() : SceProfMark{};
    long long n_head = 0, n_vc = 0;   // CG-pass launches, V-cycle invocations
    SCE_TRY(S.read_counter(&n_act));
    int total_inner = 0;

    // one CG iteration: beta from the preconditioner's r.z partials, p = z +
    // beta p, the deferred d += alpha p, q = A p (partials of p.q in part2);
    // alpha from them, r -= alpha q (partials of r.r in part), |r|^2 ...
    const int rz_nblk = S.fused ? S.rz_blocks() : l0.nblk;
    const int fold = cg_fold_mode();
    auto iter_head = [&]() -> int {
        ++n_head;
        T *pin = S.par ? S.p : S.p2, *pout = S.par ? S.p2 : S.p;
        {
            // reads cx, cy, z, p_in, d; writes p_out, d, q
            SceProf pr(KP_SPMV, st, S.vb(0, 8.0));
            if (l0.vpt == 8)
                pspmv_kernel<T, 8><<<g0, l0.tpb, 0, st>>>(S.cx[0], S.cy[0], S.z[0], pin, pout,
                                                          S.q, S.d, S.part, rz_nblk, S.sc, count,
                                                          S.par, fold, n0, 8, S.part2, l0.nblk,
                                                          S.sc.act_in);
            else
                pspmv_kernel<T><<<g0, l0.tpb, 0, st>>>(S.cx[0], S.cy[0], S.z[0], pin, pout, S.q,
                                                       S.d, S.part, rz_nblk, S.sc, count, S.par,
                                                       fold, n0, l0.vpt, S.part2, l0.nblk,
                                                       S.sc.act_in);
        }
        if (fold == FOLD_NONE) S.reduce(RED_ALPHA, S.sc.act_in, 0.0, 0.0, -1, S.par, S.part2);
        {
            SceProf pr(KP_AXPY, st, S.vb(0, 3.0));
            if (l0.vpt == 8)
                rupdate_kernel<T, 8><<<g0, l0.tpb, 0, st>>>(S.b[0], S.q, S.part2, l0.nblk, S.sc,
                                                            count, S.par, fold, n0, 8, S.part,
                                                            l0.nblk, S.sc.act_in);
            else
                rupdate_kernel<T><<<g0, l0.tpb, 0, st>>>(S.b[0], S.q, S.part2, l0.nblk, S.sc,
                                                         count, S.par, fold, n0, l0.vpt, S.part,
                                                         l0.nblk, S.sc.act_in);
        }
        SCE_CUDA(cudaMemsetAsync(S.sc.counter, 0, sizeof(int), st));
        S.reduce(RED_RR, S.sc.act_in);
        return CE_OK;
    };
    // ... and z = M^-1 r with its r.z partials, then beta (FOLD_BOTH: formed by
    // the next CG pass; the p update is part of it)
    auto iter_tail = [&]() -> int {
        ++n_vc;
        if (S.fused) {
            S.vcycle_fused(true);
        } else {
            SCE_CUDA(cudaMemsetAsync(S.z[0], 0, c0 * sizeof(T), st));
            S.vcycle(0);
            SceProf pr(KP_DOT, st, S.vb(0, 2.0));
            dot_kernel<T><<<g0, l0.tpb, 0, st>>>(S.b[0], S.z[0], n0, l0.vpt, S.part, l0.nblk,
                                                 S.sc.act_in);
        }
        if (fold != FOLD_BOTH) S.reduce(RED_BETA, S.sc.act_in, 0.0, 0.0, rz_nblk);
        S.par ^= 1;
        return CE_OK;
    };
    // CUDA graph of check_every iterations (head + tail each), captured once
    // per cached solver and replayed by every later solve of the same plan
    // (SCE_GRAPHS=1: not on the legacy default stream, during a capture or
    // with the launch profiler on).  A failed capture falls back to stream
    // launches.
    // (an even number of iterations per graph: each toggles the p array, and
    // every replay must start from the parity it was captured with)
    bool use_graph = cached && check_every % 2 == 0;
    auto capture_graph = [&]() -> int {
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return CE_ERR_CUDA;
        }
        int rc = CE_OK;
        for (int k = 0; k < check_every && rc == CE_OK; ++k) {
            rc = iter_head();
            if (rc == CE_OK) rc = iter_tail();
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(st, &g);
        if (rc != CE_OK || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return CE_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&S.graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            S.graph = nullptr;
            cudaGetLastError();
            return CE_ERR_CUDA;
        }
        return CE_OK;
    };
    for (int outer = 0; outer < 64 && n_act > 0 && total_inner < maxit; ++outer) {
        // inner PCG on the correction equation, samples with act_in set; no
        // pending d update (alpha = 0) and p_0 = z (beta = 0; folded: the r.z
        // slot of iteration -1 holds 0)
        SCE_CUDA(cudaMemsetAsync(S.d, 0, c0 * sizeof(T), st));
        SCE_CUDA(cudaMemsetAsync(S.sc.alpha, 0, (size_t)count * sizeof(double), st));
        if (sizeof(T) == 4 && fold != FOLD_NONE)
            SCE_CUDA(cudaMemsetAsync(S.sc.alphaf, 0, (size_t)count * sizeof(float), st));
        if (fold != FOLD_BOTH)
            SCE_CUDA(cudaMemsetAsync(S.sc.beta, 0, (size_t)count * sizeof(double), st));
        else if (sizeof(T) == 4)
            SCE_CUDA(cudaMemsetAsync(S.sc.rzf + count, 0, (size_t)count * sizeof(float2), st));
        else
            SCE_CUDA(cudaMemsetAsync(S.sc.rz + count, 0, (size_t)count * sizeof(double), st));
        S.par = 0;
        ++n_vc;
        if (S.fused) {
            S.vcycle_fused(true);
        } else {
            SCE_CUDA(cudaMemsetAsync(S.z[0], 0, c0 * sizeof(T), st));
            S.vcycle(0);
            SceProf pr(KP_DOT, st, S.vb(0, 2.0));
            dot_kernel<T><<<g0, l0.tpb, 0, st>>>(S.b[0], S.z[0], n0, l0.vpt, S.part, l0.nblk,
                                                 S.sc.act_in);
        }
        if (fold != FOLD_BOTH) S.reduce(RED_RZ0, S.sc.act_in, 0.0, 0.0, rz_nblk);
        int in_act = n_act;
        for (int it = 0; it < inner_max && in_act > 0 && total_inner < maxit;) {
            // four iterations as one graph launch when they fit the budgets (the
            // per-sample flags make them exact: converged samples skip every kernel)
            if (use_graph && it % check_every == 0 && it + check_every <= inner_max &&
                total_inner + check_every <= maxit) {
                if (!S.graph && capture_graph() != CE_OK) use_graph = false;
                if (use_graph) {
                    SCE_CUDA(cudaGraphLaunch(S.graph, st));
                    it += check_every;
                    total_inner += check_every;
                    SCE_TRY(S.read_counter(&in_act));
                    continue;
                }
            }
            SCE_TRY(iter_head());
            ++total_inner;
            ++it;
            if (it % check_every == 0) {
                SCE_TRY(S.read_counter(&in_act));
                if (in_act == 0) break;
            }
            SCE_TRY(iter_tail());
        }
        SCE_CUDA(cudaGetLastError());
        {
            // reads d, p and u, writes u (the last deferred CG update folded in)
            SceProf pr(KP_OUTER_UPD, st, S.vb(0, 2.0, 16.0));
            if (l0.vpt == 8)
                outer_update_kernel<T, O, 8><<<g0, l0.tpb, 0, st>>>(
                    o, S.d, S.p, S.p2, S.sc.alpha, S.sc.ppar, n0, 8, S.sc.act_out);
            else
                outer_update_kernel<T, O><<<g0, l0.tpb, 0, st>>>(
                    o, S.d, S.p, S.p2, S.sc.alpha, S.sc.ppar, n0, l0.vpt, S.sc.act_out);
        }
        {
            // reads u (8 B) and both conductances (16 B: FP64, or FP32 hi + lo), writes rin
            SceProf pr(KP_OUTER_RES, st, S.vb(0, 1.0, 24.0));
            if (l0.vpt == 8)
                outer_residual_kernel<T, O, 8><<<g0, l0.tpb, 0, st>>>(
                    o, F, n0, 8, S.b[0], S.part, l0.nblk, S.sc.act_out, row_magic(n0 + 1));
            else
                outer_residual_kernel<T, O><<<g0, l0.tpb, 0, st>>>(
                    o, F, n0, l0.vpt, S.b[0], S.part, l0.nblk, S.sc.act_out,
                    row_magic(n0 + 1));
        }
        SCE_CUDA(cudaMemsetAsync(S.sc.counter, 0, sizeof(int), st));
        S.reduce(RED_ORR, S.sc.act_out, rtol2, in_rel2);
        SCE_CUDA(cudaGetLastError());
        SCE_TRY(S.read_counter(&n_act));
    }

    // QoIs (outflow and L2 norm need a pass over the grid; the point value not)
    const bool grid_qoi = (qmask & 5) != 0;
    if (grid_qoi) {
        SceProf pr(KP_QOI, st, S.vb(0, 0.0, 16.0));
        qoi_partial_kernel<<<g0, l0.tpb, 0, st>>>(o, n0, l0.vpt, S.part, S.part2, l0.nblk,
                                                  qmask);
    }
    SCE_CUDA(cudaMemsetAsync(S.misc + 1, 0, 3 * sizeof(int), st));
    {
        // one warp per sample (launch-latency bound, like the level sums)
        SceProf pr(KP_LEVEL, st, (double)count * 64.0);
        qoi_final_kernel<<<(count * 32 + 255) / 256, 256, 0, st>>>(
            grid_qoi ? S.part : nullptr, grid_qoi ? S.part2 : nullptr, l0.nblk, count, o, n0,
            p->f, S.sc, rtol2, qoi, iters, status, S.misc + 1, qmask);
    }
    SCE_CUDA(cudaGetLastError());
    if (u_out) {
        if constexpr (mixed) {
            if (u_ff) {   // the float-float pairs as they are
                SCE_CUDA(cudaMemcpyAsync(u_out, S.uff, c0 * sizeof(float2),
                                         cudaMemcpyDeviceToDevice, st));
            } else {
                SceProf pr(KP_COPY, st, S.vb(0, 0.0, 16.0));
                u_to_double_kernel<<<g0, l0.tpb, 0, st>>>(o, n0, l0.vpt, u_out);
            }
        } else {
            SCE_CUDA(cudaMemcpyAsync(u_out, S.u64, c0 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
    }
    int hm[3] = {0, 0, 0};
    SCE_CUDA(cudaMemcpyAsync(hm, S.misc + 1, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    SCE_CUDA(cudaStreamSynchronize(st));
    if (n_failed_out) *n_failed_out = hm[0];
    if (max_iters_out) {
        max_iters_out[0] = hm[1];
        max_iters_out[1] = hm[2];
    }
    if (sce_prof_on() && count > 0) {
        // an active sample runs one CG pass, one r update and one V-cycle per
        // iteration (the V-cycle at an inner solve's start stands in for the
        // one its last iteration skips), so the passes that ran are the
        // samples' total iteration count hm[2]
        static const int cg_ids[] = {KP_SPMV, KP_AXPY};
        static const int vc_ids[] = {KP_MG_DOWN, KP_MG_UP, KP_MG_DOWN3, KP_MG_UP3, KP_MG_V64,
                                     KP_MG_TAIL, KP_SMOOTH, KP_RESTRICT, KP_PROLONG,
                                     KP_COARSEST, KP_DOT};
        if (n_head > 0)
            sce_prof_scale(prof_mark, st, cg_ids, 2,
                           std::min(1.0, (double)hm[2] / ((double)n_head * count)));
        if (n_vc > 0)
            sce_prof_scale(prof_mark, st, vc_ids, (int)(sizeof(vc_ids) / sizeof(vc_ids[0])),
                           std::min(1.0, (double)hm[2] / ((double)n_vc * count)));
    }
    lease.ok = true;
    return hm[0] > 0 ? CE_ERR_NOT_CONVERGED : CE_OK;
}

}  // namespace

extern "C" int darcy_solver_cache_clear(void *stream) {
    const cudaStream_t st = as_stream(stream);
    const int a = solver_pool<float>().clear(st);
    const int b = solver_pool<double>().clear(st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CE_ERR_CUDA;
    return a != CE_OK ? a : b;
}

int sce_darcy_solve_impl(const darcy_problem *p, const void *k, int count, double *qoi, int *iters,
                         int *status, double *u_out, cudaStream_t st, int *max_iters_out,
                         int *n_failed_out, int qmask, const double *u_init, bool u_ff) {
    if (!p || !k || !qoi || count < 0) return CE_ERR_INVALID_ARG;
    if (!is_pow2(p->n) || p->n < 4 || p->n > 4096) return CE_ERR_INVALID_ARG;
    if (p->precision != 32 && p->precision != 64) return CE_ERR_INVALID_ARG;
    if (!(p->rtol > 0) || count > 65535) return CE_ERR_INVALID_ARG;
    if (count == 0) return CE_OK;
    qmask &= 7;
    if (u_ff && p->precision != 32) return CE_ERR_INVALID_ARG;
    if (p->precision == 32 && p->n <= sce_small_max_n() && p->n <= 64)
        return sce_darcy_small(p, (const float *)k, count, qoi, iters, status, u_out, st,
                               max_iters_out, n_failed_out, qmask | (u_ff ? 8 : 0), u_init,
                               u_ff);
    if (p->precision == 64)
        return darcy_solve_t<double, double>(p, (const double *)k, count, qoi, iters, status,
                                             u_out, st, max_iters_out, n_failed_out, qmask,
                                             u_init, false);
    return darcy_solve_t<float, float>(p, (const float *)k, count, qoi, iters, status, u_out, st,
                                       max_iters_out, n_failed_out, qmask, u_init, u_ff);
}

extern "C" int darcy_solve_batch(const darcy_problem *p, const void *k, int count, double *qoi,
                                 int *iters, int *status, double *u_out, void *stream) {
    return sce_darcy_solve_impl(p, k, count, qoi, iters, status, u_out, as_stream(stream), nullptr,
                                nullptr, 7);
}

// ---------------------------------------------------------------- tile tuner
namespace {
// A smooth synthetic coefficient for timing: k = exp(0.8 sin(6 pi x) cos(4 pi y)
// + 0.1 (s mod 7)), per sample s; the timings compare window heights at equal
// iteration counts (every height computes the same iterates up to rounding).
template <typename T>
__global__ void tuner_field_kernel(T *k, int n, int count) {
    const long long V = (long long)(n + 1) * (n + 1);
    const long long tot = V * count;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
         q += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(q / V);
        const int v = (int)(q - (long long)s * V);
        const int j = v / (n + 1), i = v - j * (n + 1);
        const double x = (double)i / n, y = (double)j / n;
        k[q] = (T)exp(0.8 * sin(6.0 * M_PI * x) * cos(4.0 * M_PI * y) + 0.1 * (s % 7));
    }
}
}  // namespace

extern "C" int darcy_autotune_tiles(int n, int precision, int count, int reps, void *stream,
                                    int *height) {
    if (n < 128 || n > 4096 || !is_pow2(n) || (precision != 32 && precision != 64) ||
        count <= 0 || count > 65535 || reps <= 0)
        return CE_ERR_INVALID_ARG;
    const cudaStream_t st = as_stream(stream);
    const int tsize = precision == 64 ? 8 : 4;
    const long long V = (long long)(n + 1) * (n + 1);
    void *k = nullptr;
    double *qoi = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto release = [&]() {
        if (k) sce_free(k, st);
        if (qoi) sce_free(qoi, st);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    };
    int rc = sce_alloc(&k, (size_t)count * V * tsize, st);
    if (rc == CE_OK) rc = sce_alloc((void **)&qoi, (size_t)count * 3 * sizeof(double), st);
    if (rc != CE_OK) {
        release();
        return rc;
    }
    if (precision == 64) tuner_field_kernel<double><<<1024, 256, 0, st>>>((double *)k, n, count);
    else tuner_field_kernel<float><<<1024, 256, 0, st>>>((float *)k, n, count);
    if (cudaGetLastError() != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess) {
        release();
        return CE_ERR_CUDA;
    }
    const darcy_problem p{n, 1.0, 1e-8, 1000, precision};
    int best = MG_SH;
    float best_ms = 0.0f;
    for (int h : kTileHeights) {
        {
            std::lock_guard<std::mutex> lk(g_tile_mu);
            g_tile_sh[{tsize, n}] = h;
        }
        float ms_min = 0.0f;
        for (int r = 0; r <= reps; ++r) {   // the first call warms up
            if (cudaEventRecord(a, st) != cudaSuccess) rc = CE_ERR_CUDA;
            if (rc == CE_OK)
                rc = sce_darcy_solve_impl(&p, k, count, qoi, nullptr, nullptr, nullptr, st, nullptr,
                                          nullptr, 7);
            if (rc == CE_ERR_NOT_CONVERGED) rc = CE_OK;
            float ms = 0.0f;
            if (rc == CE_OK && (cudaEventRecord(b, st) != cudaSuccess ||
                                cudaEventSynchronize(b) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
                rc = CE_ERR_CUDA;
            if (rc != CE_OK) break;
            if (r > 0 && (r == 1 || ms < ms_min)) ms_min = ms;
        }
        if (rc != CE_OK) break;
        if (h == kTileHeights[0] || ms_min < best_ms) {
            best_ms = ms_min;
            best = h;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        g_tile_sh[{tsize, n}] = rc == CE_OK ? best : MG_SH;
    }
    release();
    if (rc == CE_OK && height) *height = best;
    return rc;
}


// Fused, shared-memory-tiled multigrid kernels for the batched solver.
//
// The fine grid of a level is partitioned by tiles of CW x CH coarse vertices;
// tile (tx, ty) owns the fine vertices [2 I0, 2 I0 + 2 CW) x [2 J0, 2 J0 + 2 CH)
// (I0 = tx CW, J0 = ty CH), so the owned regions of all tiles cover the fine
// grid exactly once and the coarse tiles cover the coarse grid exactly once.
// Each kernel stages a 64 x 32 window (owned region plus halo) in shared
// memory, recomputes halo values instead of exchanging them, and writes only
// what it owns.  Thread (x, y) of the 32 x 8 block handles the window
// elements (x + 32 a, y + 8 b), a < 2, b < MG_SH / 8, so no index arithmetic
// is repeated per pass; 1/diag is computed once per element.
//
//   mg_down: pre-smoothing from a zero guess (red then black Gauss-Seidel),
//            fine residual, full-weighting restriction -> zpre (fine), b (coarse).
//            After the black half-sweep the residual vanishes at the black
//            vertices (each was just solved for with its red neighbours
//            fixed), so it is formed at the red vertices only and the
//            restriction sums the coarse vertex and its four diagonal
//            neighbours (the red ones of its 3 x 3 stencil).
//   mg_up  : z = zpre + bilinear prolongation of the coarse correction, then
//            post-smoothing (black then red) -> z (fine); optionally the
//            partial sums of r . z (level 0, for CG's beta).  zpre and z are
//            distinct arrays: a tile reads zpre in its halo, which other
//            tiles of the same launch own and write to z.
//   mg_tail: the whole V-cycle of the coarse levels n <= NT_N of one sample in
//            one thread block (shared memory)
// Together with the exact coarsest solve this is the same symmetric V(1,1)
// cycle as the level-by-level kernels (up to rounding: 1/diag is applied as a
// reciprocal multiply).
#pragma once

#include "block_mg.cuh"
#include "stencil.cuh"

namespace sce {

#ifndef SCE_MG_SH
#define SCE_MG_SH 32
#endif
constexpr int MG_SW = 64;                  // window width (= row stride)
constexpr int MG_SH = SCE_MG_SH;           // window height (multiple of 8)
constexpr int MG_CW = (MG_SW - 6) / 2;     // 29 coarse vertices per tile in x
constexpr int MG_CH = (MG_SH - 6) / 2;     // coarse vertices per tile in y
constexpr int MG_THREADS = 256;
constexpr int MG_ROWS = MG_SH / 8;         // row groups per thread
constexpr int MG_NE = 2 * MG_ROWS;         // window elements per thread
static_assert(MG_SH % 8 == 0 && MG_NE <= 32, "tile height");
constexpr int MG_BLOCKS_PER_SM = MG_SH <= 32 ? 5 : (MG_SH <= 48 ? 3 : 2);
constexpr int MG_CCW = MG_CW + 3;          // coarse window of mg_up
constexpr int MG_CCH = MG_CH + 3;

template <typename T>
constexpr size_t mg_tile_smem_bytes() {
    return sizeof(T) * (5 * (size_t)MG_SW * MG_SH + (size_t)MG_CCW * MG_CCH);
}

template <typename T>
__device__ __forceinline__ T block_sum_t(T val, T *sh) {
    for (int o = 16; o > 0; o >>= 1) val += __shfl_down_sync(0xffffffffu, val, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = val;
    __syncthreads();
    T tot = T(0);
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += sh[i];
    return tot;
}

template <typename T> __device__ __forceinline__ T recip(T d);
template <> __device__ __forceinline__ float recip<float>(float d) { return __frcp_rn(d); }
template <> __device__ __forceinline__ double recip<double>(double d) { return 1.0 / d; }

// Gauss-Seidel update of the vertices of colour `color` ((gi + gj) % 2) in the
// local box [lo, hix] x [lo, hiy] of the window.  Lane x of warp y handles the
// column pair (2x, 2x+1) of rows y + 8b, i.e. exactly the one element of each
// pair that has the colour, so no lane idles.
template <typename T>
__device__ __forceinline__ void tile_color_pass(T *sz, const T *sb, const T *scx, const T *scy,
                                                const T *sinv, int ox, int oy, int n, int color,
                                                int lo, int hix, int hiy) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // rows ty + 8 bb all have the parity of ty: the column is the same for all bb
    const int li = 2 * tx + ((ox + oy + ty + color) & 1);
    const int gi = ox + li;
    if (li < lo || li > hix || gi < 1 || gi > n - 1) return;
#pragma unroll
    for (int bb = 0; bb < MG_ROWS; ++bb) {
        const int lj = ty + 8 * bb;
        if (lj < lo || lj > hiy) continue;
        const int gj = oy + lj;
        if (gj < 0 || gj > n) continue;
        const int l = lj * MG_SW + li;
        sz[l] = (sb[l] + scx[l - 1] * sz[l - 1] + scx[l] * sz[l + 1] +
                 scy[l - MG_SW] * sz[l - MG_SW] + scy[l] * sz[l + MG_SW]) * sinv[l];
    }
}

// Residual b - A z at the red vertices ((gi + gj) even) of the local box
// [3, MG_SW-3] x [3, MG_SH-3], in place of b; 0 at Dirichlet vertices.
template <typename T>
__device__ __forceinline__ void tile_red_residual(const T *sz, T *sb, const T *scx,
                                                  const T *scy, int ox, int oy, int n) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int li = 2 * tx + ((ox + oy + ty) & 1);
    const int gi = ox + li;
    if (li < 3 || li > MG_SW - 3) return;
    const bool unk_x = gi >= 1 && gi <= n - 1;
#pragma unroll
    for (int bb = 0; bb < MG_ROWS; ++bb) {
        const int lj = ty + 8 * bb;
        if (lj < 3 || lj > MG_SH - 3) continue;
        const int gj = oy + lj;
        const int l = lj * MG_SW + li;
        T rv = T(0);
        if (unk_x && gj >= 0 && gj <= n) {
            const T zc = sz[l];
            rv = sb[l] - (scx[l - 1] * (zc - sz[l - 1]) + scx[l] * (zc - sz[l + 1]) +
                          scy[l - MG_SW] * (zc - sz[l - MG_SW]) + scy[l] * (zc - sz[l + MG_SW]));
        }
        sb[l] = rv;
    }
}

// Element e (0..7) of this thread: local (li, lj) and offset in the window.
#define MG_ELEM(e, li, lj, l)                                   \
    const int li = (threadIdx.x & 31) + 32 * ((e) & 1);         \
    const int lj = (threadIdx.x >> 5) + 8 * ((e) >> 1);         \
    const int l = lj * MG_SW + li

template <typename T>
__global__ void __launch_bounds__(MG_THREADS, MG_BLOCKS_PER_SM) mg_down_kernel(
    const T *__restrict__ cx, const T *__restrict__ cy, const T *__restrict__ b,
    T *__restrict__ zpre, int n, T *__restrict__ bc, int tiles_x, const int *__restrict__ act) {
    constexpr int LS = MG_SW * MG_SH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sb = reinterpret_cast<T *>(smem_raw);
    T *scx = sb + LS, *scy = scx + LS, *sz = scy + LS, *sinv = sz + LS;
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int nc = n / 2, w = n + 1, wc = nc + 1;
    const long long V = (long long)w * w, Vc = (long long)wc * wc;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int I0 = tx * MG_CW, J0 = ty * MG_CH;
    const int ox = 2 * I0 - 4, oy = 2 * J0 - 4;
    const T *bs = b + s * V, *xs = cx + s * V, *ys = cy + s * V;
    unsigned unk = 0;   // bit e: element e is an unknown of the grid
#pragma unroll
    for (int e = 0; e < MG_NE; ++e) {
        MG_ELEM(e, li, lj, l);
        const int gi = ox + li, gj = oy + lj;
        const bool in = gi >= 0 && gi <= n && gj >= 0 && gj <= n;
        const int g = gj * w + gi;
        sb[l] = in ? bs[g] : T(0);
        scx[l] = in ? xs[g] : T(0);
        scy[l] = in ? ys[g] : T(0);
        if (in && gi >= 1 && gi <= n - 1) unk |= 1u << e;
    }
    __syncthreads();
    // 1/diag; red from z = 0: z = b / diag
#pragma unroll
    for (int e = 0; e < MG_NE; ++e) {
        MG_ELEM(e, li, lj, l);
        T inv = T(0), zv = T(0);
        if (li >= 1 && lj >= 1 && ((unk >> e) & 1)) {
            inv = recip(scx[l - 1] + scx[l] + scy[l - MG_SW] + scy[l]);
            if (!(((ox + li) + (oy + lj)) & 1)) zv = sb[l] * inv;
        }
        sinv[l] = inv;
        sz[l] = zv;
    }
    __syncthreads();
    // black on local [2, SW-2] x [2, SH-2]
    tile_color_pass(sz, sb, scx, scy, sinv, ox, oy, n, 1, 2, MG_SW - 2, MG_SH - 2);
    __syncthreads();
    tile_red_residual(sz, sb, scx, scy, ox, oy, n);
    __syncthreads();
    // restriction to the tile's coarse vertices (red stencil points only)
    T *bcs = bc + s * Vc;
    for (int c = threadIdx.x; c < MG_CW * MG_CH; c += MG_THREADS) {
        const int ci = c % MG_CW, cj = c / MG_CW;
        const int I = I0 + ci, J = J0 + cj;
        if (I > nc || J > nc) continue;
        T acc = T(0);
        if (I > 0 && I < nc) {
            const int l0 = (2 * cj + 4) * MG_SW + 2 * ci + 4;
            acc = T(0.25) * (sb[l0 - MG_SW - 1] + sb[l0 - MG_SW + 1] + sb[l0 + MG_SW - 1] +
                             sb[l0 + MG_SW + 1]) +
                  sb[l0];
        }
        bcs[J * wc + I] = acc;
    }
    // owned fine vertices: local [4, 4 + 2 CW) x [4, 4 + 2 CH)
    T *zs = zpre + s * V;
#pragma unroll
    for (int e = 0; e < MG_NE; ++e) {
        MG_ELEM(e, li, lj, l);
        if (li < 4 || li >= 4 + 2 * MG_CW || lj < 4 || lj >= 4 + 2 * MG_CH) continue;
        const int gi = ox + li, gj = oy + lj;
        if (gi > n || gj > n) continue;
        zs[gj * w + gi] = sz[l];
    }
}

template <typename T>
__global__ void __launch_bounds__(MG_THREADS, MG_BLOCKS_PER_SM) mg_up_kernel(
    const T *__restrict__ cx, const T *__restrict__ cy, const T *__restrict__ b,
    const T *__restrict__ zpre, T *__restrict__ z, int n, const T *__restrict__ zc, int tiles_x,
    const int *__restrict__ act, double *__restrict__ part_rz, int nblk) {
    constexpr int LS = MG_SW * MG_SH;
    constexpr int UW = 2 * MG_CW + 4, UH = 2 * MG_CH + 4;   // used window: 62 x 30
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T sred[32];
    T *sb = reinterpret_cast<T *>(smem_raw);
    T *scx = sb + LS, *scy = scx + LS, *sz = scy + LS, *sinv = sz + LS, *szc = sinv + LS;
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int nc = n / 2, w = n + 1, wc = nc + 1;
    const long long V = (long long)w * w, Vc = (long long)wc * wc;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int I0 = tx * MG_CW, J0 = ty * MG_CH;
    const int ox = 2 * I0 - 2, oy = 2 * J0 - 2;
    const int cox = I0 - 1, coy = J0 - 1;
    const T *bs = b + s * V, *xs = cx + s * V, *ys = cy + s * V, *zcs = zc + s * Vc;
    const T *zps = zpre + s * V;
    T *zs = z + s * V;
    for (int c = threadIdx.x; c < MG_CCW * MG_CCH; c += MG_THREADS) {
        const int ci = c % MG_CCW, cj = c / MG_CCW;
        const int I = cox + ci, J = coy + cj;
        szc[c] = (I >= 0 && I <= nc && J >= 0 && J <= nc) ? zcs[J * wc + I] : T(0);
    }
    unsigned unk = 0;
#pragma unroll
    for (int e = 0; e < MG_NE; ++e) {
        MG_ELEM(e, li, lj, l);
        const int gi = ox + li, gj = oy + lj;
        const bool in = li < UW && lj < UH && gi >= 0 && gi <= n && gj >= 0 && gj <= n;
        const int g = gj * w + gi;
        sb[l] = in ? bs[g] : T(0);
        scx[l] = in ? xs[g] : T(0);
        scy[l] = in ? ys[g] : T(0);
        sz[l] = in ? zps[g] : T(0);
        if (in && gi >= 1 && gi <= n - 1) unk |= 1u << e;
    }
    __syncthreads();
    // 1/diag and z += P zc at every unknown of the used window
#pragma unroll
    for (int e = 0; e < MG_NE; ++e) {
        MG_ELEM(e, li, lj, l);
        if (!((unk >> e) & 1)) {
            sinv[l] = T(0);
            continue;
        }
        sinv[l] = (li >= 1 && lj >= 1) ? recip(scx[l - 1] + scx[l] + scy[l - MG_SW] + scy[l]) : T(0);
        const int gi = ox + li, gj = oy + lj;
        const int c = ((gj >> 1) - coy) * MG_CCW + ((gi >> 1) - cox);
        // bilinear weights: (1, 0) on even fine indices, (1/2, 1/2) on odd ones
        const T wx1 = (gi & 1) ? T(0.5) : T(0), wy1 = (gj & 1) ? T(0.5) : T(0);
        const T wx0 = T(1) - wx1, wy0 = T(1) - wy1;
        sz[l] += wy0 * (wx0 * szc[c] + wx1 * szc[c + 1]) +
                 wy1 * (wx0 * szc[c + MG_CCW] + wx1 * szc[c + MG_CCW + 1]);
    }
    __syncthreads();
    // black on local [1, UW-2] x [1, UH-2], then red on [2, UW-3] x [2, UH-3]
    tile_color_pass(sz, sb, scx, scy, sinv, ox, oy, n, 1, 1, UW - 2, UH - 2);
    __syncthreads();
    tile_color_pass(sz, sb, scx, scy, sinv, ox, oy, n, 0, 2, UW - 3, UH - 3);
    __syncthreads();
    // owned fine vertices: local [2, 2 + 2 CW) x [2, 2 + 2 CH)
    T rz = T(0);
#pragma unroll
    for (int e = 0; e < MG_NE; ++e) {
        MG_ELEM(e, li, lj, l);
        if (li < 2 || li >= 2 + 2 * MG_CW || lj < 2 || lj >= 2 + 2 * MG_CH) continue;
        const int gi = ox + li, gj = oy + lj;
        if (gi > n || gj > n) continue;
        zs[gj * w + gi] = sz[l];
        rz += sb[l] * sz[l];
    }
    if (part_rz) {
        const T tot = block_sum_t(rz, sred);
        if (threadIdx.x == 0) part_rz[(long long)s * nblk + blockIdx.x] = (double)tot;
    }
}

#undef MG_ELEM

struct TailPtrs {
    void *cx[8], *cy[8];
};

// V-cycle of levels NT_N, NT_N/2, ..., 2 of one sample per block.
template <typename T, int NT_N, int NTHR>
__global__ void __launch_bounds__(NTHR) mg_tail_kernel(TailPtrs tp, const T *__restrict__ b,
                                                       T *__restrict__ z,
                                                       const int *__restrict__ act,
                                                       double *__restrict__ part_rz) {
    using Lay = MGPackedLayout<NT_N>;
    constexpr int NL = mg_levels(NT_N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T sred[32];
    const int s = blockIdx.x;
    if (!act[s]) return;
    T *base = reinterpret_cast<T *>(smem_raw);
#pragma unroll
    for (int L = 0; L < NL; ++L) {
        const int VL = mg_vof(NT_N >> L);
        T *cx = base + Lay::off(L, 0), *cy = base + Lay::off(L, 1);
        const T *gx = reinterpret_cast<const T *>(tp.cx[L]) + (long long)s * VL;
        const T *gy = reinterpret_cast<const T *>(tp.cy[L]) + (long long)s * VL;
        for (int v = threadIdx.x; v < VL; v += NTHR) {
            cx[v] = gx[v];
            cy[v] = gy[v];
        }
    }
    constexpr int V0 = (NT_N + 1) * (NT_N + 1);
    const T *bs = b + (long long)s * V0;
    T *b0 = base + Lay::off(0, 2), *z0 = base + Lay::off(0, 3);
    for (int v = threadIdx.x; v < V0; v += NTHR) b0[v] = bs[v];
    __syncthreads();
    block_vcycle<T, NT_N, NTHR, Lay>(base);
    T *zs = z + (long long)s * V0;
    T rz = T(0);
    for (int v = threadIdx.x; v < V0; v += NTHR) {
        zs[v] = z0[v];
        rz += b0[v] * z0[v];
    }
    if (part_rz) {
        const T tot = block_sum_t(rz, sred);
        if (threadIdx.x == 0) part_rz[s] = (double)tot;
    }
}

template <typename T, int NT_N>
constexpr size_t tail_smem_bytes() {
    size_t t = 0;
    for (int n = NT_N; n >= 2; n /= 2) t += 4 * (size_t)(n + 1) * (n + 1);
    return t * sizeof(T);
}

}  // namespace sce

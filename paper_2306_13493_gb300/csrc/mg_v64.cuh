// One multigrid V-cycle of a whole n = 64 grid and of the levels below it, one
// sample per thread block: NUT sweeps per side on the n = 64 level, NUS on each
// level below it.
//
// The 65 x 65 fine grid has 63 unknown columns (1..63) between its two
// Dirichlet columns, so its columns 0..63 fit one 64-wide register window
// exactly: no halo, no overlapping tiles.  17 warps hold rows [4 w, 4 w + 4)
// (68 rows, the last three outside the grid), lane x the columns (2 x, 2 x + 1),
// with the register layout, the shuffles and the strip exchange of the tiled
// kernels (mg_tiles.cuh).  The east neighbour of column 63 is the Dirichlet
// column 64, whose z is 0 (EAST0).  Elements outside the grid hold zero data
// and 1/diag = 0, as in the tiles.
//
//   load b, cx, cy of the level and the conductances of levels 32..2
//   pre-smoothing from z = 0 (NUT sweeps: red, then black), red residuals, full-weighting
//   restriction into the b of level 32 in shared memory
//   V-cycle of levels 32..2 in shared memory (block_vcycle, NUS sweeps per side)
//   bilinear prolongation of the level-32 correction, post-smoothing (NUT
//   sweeps: black, then red), z of the level to global memory, optionally the block's
//   partial sum of b . z (CG's beta when the level is the finest)
//
// The arithmetic per vertex is that of mg_down / mg_tail / mg_up, so this is
// the same symmetric cycle; it replaces their three launches on this level by
// one and the 2.8-fold window overlap of 64 x 32 tiles on a 65 x 65 grid by
// none.
#pragma once

#include "mg_tiles.cuh"

namespace sce {

constexpr int V64_N = 64;
constexpr int V64_NW = 17;                      // 68 rows >= 65
constexpr int V64_THREADS = 32 * V64_NW;        // 544
// levels 32..2 in shared memory (PAD: level 32 in rows of 34, see mg_pitch)
template <bool PAD>
using V64Lay = MGPackedLayout<V64_N / 2, PAD>;

template <typename T, bool PAD = false>
constexpr size_t v64_smem_bytes() {
    return sizeof(T) * ((size_t)V64Lay<PAD>::total() + 2 * 2 * V64_NW * (size_t)MG_SW +
                        V64_NW * (size_t)MG_SW + 32 + tile_inv_slots(V64_NW));
}

// tp.cx[i], tp.cy[i]: conductances of level 32 >> i (i = 0..4), per sample
// contiguous.  part_rz: one slot per sample, or NULL.  WARP_N > 0: the levels
// of at most WARP_N cells run on warp 0 alone (see block_vcycle_from).
// NUT: sweeps per side on the n = 64 level, NUS on the levels 32..2 in shared
// memory; PAD: their layout.
template <typename T, int WARP_N = 0, int NUT = mg_nu<T>(), int NUS = mg_nu<T>(),
          bool PAD = false>
__global__ void __launch_bounds__(V64_THREADS, 2) mg_v64_kernel(
    const T *__restrict__ cx, const T *__restrict__ cy, const T *__restrict__ b,
    T *__restrict__ z, TailPtrs tp, const int *__restrict__ act, double *__restrict__ part_rz) {
    using Lay = V64Lay<PAD>;
    constexpr int NC = V64_N / 2, W = V64_N + 1, PC = Lay::pitch(0);   // PC: level 32's row pitch
    constexpr int V = W * W;
    constexpr int NL = mg_levels(NC);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *base = reinterpret_cast<T *>(smem_raw);
    T *xz = base + Lay::total();
    T *xrow = xz + 2 * 2 * V64_NW * MG_SW;
    T *sred = xrow + V64_NW * MG_SW;
    T *sinv = sred + 32;   // the threads' 1/diag slices
    const int s = blockIdx.x;
    if (!act[s]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // conductances of the coarse levels (read by block_vcycle after the barriers below)
#pragma unroll
    for (int L = 0; L < NL; ++L) {
        const int VL = mg_vof(NC >> L), wl = (NC >> L) + 1, pl = Lay::pitch(L);
        T *sx = base + Lay::off(L, 0), *sy = base + Lay::off(L, 1);
        const T *gx = reinterpret_cast<const T *>(tp.cx[L]) + (long long)s * VL;
        const T *gy = reinterpret_cast<const T *>(tp.cy[L]) + (long long)s * VL;
        for (int v = threadIdx.x; v < VL; v += V64_THREADS) {
            const int J = v / wl, q = J * pl + (v - J * wl);
            sx[q] = gx[v];
            sy[q] = gy[v];
        }
    }

    // the lane's 2 x 4 block: columns 2 lane + c, rows 4 warp + r (rows <= 64 in the grid)
    TileBlock<T> t;
    const int gi0 = 2 * lane, gj0 = 4 * warp;
    const T *bs = b + (long long)s * V, *xs = cx + (long long)s * V, *ys = cy + (long long)s * V;
    unsigned unk = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int e = 2 * r + c, gi = gi0 + c, gj = gj0 + r;
            const bool in = gj <= V64_N;
            const int g = gj * W + gi;
            t.b[e] = in ? bs[g] : T(0);
            t.cxe[e] = in ? xs[g] : T(0);
            t.cyn[e] = in ? ys[g] : T(0);
            if (in && gi >= 1) unk |= 1u << e;
        }
    }
    tile_diag<T, V64_NW>(t, xrow, lane, warp, unk, sinv);

    // pre-smoothing: red from z = 0, then black
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int e = 2 * r + c;
            t.z[e] = ((c + r) & 1) == 0 ? t.b[e] * tile_inv(t, c, r) : T(0);
        }
    }
    tile_exchange<T, V64_NW>(t, xz, 0, lane, warp);
    tile_half_sweep<T, 1, 0, true>(t);
    tile_exchange<T, V64_NW>(t, xz, 1, lane, warp);
#pragma unroll
    for (int k = 1; k < NUT; ++k) {   // the further sweeps: red, black
        tile_half_sweep<T, 0, 0, true>(t);
        tile_exchange<T, V64_NW>(t, xz, 0, lane, warp);
        tile_half_sweep<T, 1, 0, true>(t);
        tile_exchange<T, V64_NW>(t, xz, 1, lane, warp);
    }

    // red residuals (the black ones vanish) and full weighting: coarse vertex
    // (lane, 2 warp + k) sits at (c = 0, r = 2 k); its diagonal neighbours are
    // the red elements of rows 2k - 1 and 2k + 1, columns 2 lane -/+ 1
    const T r0 = tile_red_residual<T, 0, true>(t, unk), r1 = tile_red_residual<T, 1, true>(t, unk);
    const T r2 = tile_red_residual<T, 2, true>(t, unk), r3 = tile_red_residual<T, 3, true>(t, unk);
    xrow[warp * MG_SW + lane] = r3;
    __syncthreads();
    const T rm = warp > 0 ? xrow[(warp - 1) * MG_SW + lane] : T(0);
    const T l1 = __shfl_up_sync(MG_FULL, r1, 1), l3 = __shfl_up_sync(MG_FULL, r3, 1);
    const T lm = __shfl_up_sync(MG_FULL, rm, 1);
    const T acc[2] = {T(0.25) * (lm + rm + l1 + r1) + r0, T(0.25) * (l1 + r1 + l3 + r3) + r2};
    T *bc = base + Lay::off(0, 2);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int J = 2 * warp + k;
        if (J <= NC) bc[J * PC + lane] = lane > 0 ? acc[k] : T(0);
    }
    if (threadIdx.x <= NC) bc[threadIdx.x * PC + NC] = T(0);   // Dirichlet column I = 32

    // levels 32..2 (block_vcycle zeroes z of level 32 and synchronises first)
    block_vcycle<T, NC, V64_THREADS, Lay, WARP_N, NUS>(base);

    // z += P zc: coarse columns lane, lane + 1 and rows 2 warp + {0, 1, 2}
    // (rows beyond 32 only feed elements outside the grid: read as 0)
    const T *zc = base + Lay::off(0, 3);
    const int J0 = 2 * warp;
    const T a0 = zc[J0 * PC + lane], a1 = zc[J0 * PC + lane + 1];
    const T b0 = J0 + 1 <= NC ? zc[(J0 + 1) * PC + lane] : T(0);
    const T b1 = J0 + 1 <= NC ? zc[(J0 + 1) * PC + lane + 1] : T(0);
    const T c0 = J0 + 2 <= NC ? zc[(J0 + 2) * PC + lane] : T(0);
    const T c1 = J0 + 2 <= NC ? zc[(J0 + 2) * PC + lane + 1] : T(0);
    const T h = T(0.5), qq = T(0.25);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!((unk >> k) & 1)) continue;
        const int r = k >> 1, c = k & 1;
        T pv;
        const T x0 = r < 2 ? a0 : b0, x1 = r < 2 ? a1 : b1;   // coarse row J0 (+1)
        const T y0 = r < 2 ? b0 : c0, y1 = r < 2 ? b1 : c1;   // the row above it
        if ((r & 1) == 0) pv = c == 0 ? x0 : h * (x0 + x1);
        else pv = c == 0 ? h * (x0 + y0) : qq * ((x0 + x1) + (y0 + y1));
        t.z[k] += pv;
    }

    // post-smoothing: black, then red (NUT times)
#pragma unroll
    for (int k = 0; k < NUT; ++k) {
        tile_exchange<T, V64_NW>(t, xz, 0, lane, warp);
        tile_half_sweep<T, 1, 0, true>(t);
        tile_exchange<T, V64_NW>(t, xz, 1, lane, warp);
        tile_half_sweep<T, 0, 0, true>(t);
    }

    // z of the level (column 64, the Dirichlet column, is 0) and b . z
    T *zs = z + (long long)s * V;
    T rz = T(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int gj = gj0 + r;
        if (gj > V64_N) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            zs[gj * W + gi0 + c] = t.z[2 * r + c];
            rz += t.b[2 * r + c] * t.z[2 * r + c];
        }
        if (lane == 31) zs[gj * W + V64_N] = T(0);
    }
    if (part_rz) {
        const T tot = block_sum_t(rz, sred);
        if (threadIdx.x == 0) part_rz[s] = (double)tot;
    }
}

}  // namespace sce

// Fused, register-blocked multigrid kernels for the batched solver.
//
// The fine grid of a level is partitioned by tiles of CW x CH coarse vertices;
// tile (tx, ty) owns the fine vertices [2 I0, 2 I0 + 2 CW) x [2 J0, 2 J0 + 2 CH)
// (I0 = tx CW, J0 = ty CH), so the owned regions of all tiles cover the fine
// grid exactly once and the coarse tiles cover the coarse grid exactly once.
// Each kernel works on a 64 x 32 window (owned region plus halo), recomputes
// halo values instead of exchanging them with other tiles, and writes only
// what it owns.  The window lives in registers: warp w holds rows
// [4 w, 4 w + 4), lane x the columns (2 x, 2 x + 1) of them, i.e. a 2 x 4
// block per lane.  Horizontal neighbours come from the lanes beside (warp
// shuffles), vertical ones from the lane's own block except across the
// warps' strip boundaries, whose rows go through shared memory (double
// buffered, one barrier per half-sweep).  The window origin is even in both
// directions, so the colour of block element (c, r) is (c + r) % 2 for every
// lane and every loop over a colour unrolls with compile-time register
// indices.  Elements outside the grid hold zero data; at Dirichlet columns and
// outside the grid 1/diag is 0, so their z stays 0.
//
//   mg_down: pre-smoothing from a zero guess (NU sweeps of red then black
//            Gauss-Seidel), fine residual, full-weighting restriction -> zpre
//            (fine), b (coarse).
//            After the black half-sweep the residual vanishes at the black
//            vertices (each was just solved for with its red neighbours
//            fixed), so it is formed at the red vertices only and the
//            restriction sums the coarse vertex and its four diagonal
//            neighbours (the red ones of its 3 x 3 stencil).
//   mg_up  : z = zpre + bilinear prolongation of the coarse correction, then
//            post-smoothing (NU sweeps of black then red) -> z (fine); optionally the
//            partial sums of r . z (level 0, for CG's beta).  zpre and z are
//            distinct arrays: a tile reads zpre in its halo, which other
//            tiles of the same launch own and write to z.
//   mg_tail: the whole V-cycle of the coarse levels n <= NT_N of one sample in
//            one thread block (shared memory)
// Together with the exact coarsest solve this is the same symmetric
// V(nu, nu) cycle as the level-by-level kernels (up to rounding: 1/diag
// is applied as a reciprocal multiply).
#pragma once

#include "block_mg.cuh"
#include "stencil.cuh"

namespace sce {

constexpr int MG_SW = 64;                  // window width: 32 lanes x 2 columns
#ifndef SCE_MG_SH
#define SCE_MG_SH 32
#endif
constexpr int MG_SH = SCE_MG_SH;           // window height: MG_SH / 4 warps x 4 rows
#ifndef SCE_TILE_WARPS_PER_SM
#define SCE_TILE_WARPS_PER_SM 40
#endif
constexpr int MG_NW = MG_SH / 4;           // warps per block
// Halo of the windows.  In a window, every half-sweep after the first makes
// one more ring at its edges invalid (the values beyond the window are not
// there), and so do the residual and the restriction's diagonal neighbours:
// with NU sweeps per side, mg_down's window starts 2 NU + 2 fine vertices below
// and left of its owned region, mg_up's 2 NU; the owned region is 2 CW x 2 CH
// fine vertices with CW = 32 - 2 NU - 1 (29 for V(1,1), 27 for V(2,2), 25 for
// V(3,3)) and CH = SH / 2 - 2 NU - 1 for a window of SH rows.  NU is chosen per
// level by the solver (sweeps of the level's cycle), mg_nu<T>() by default.
template <typename T, int NU_ = mg_nu<T>()>
struct MGGeom {
    static_assert(NU_ >= 1 && NU_ <= 3, "sweeps per side");
    static constexpr int NU = NU_;
    static constexpr int OD = 2 * NU + 2;            // mg_down window origin: 2 I0 - OD
    static constexpr int OU = 2 * NU;                // mg_up window origin: 2 I0 - OU
    static constexpr int CW = MG_SW / 2 - 2 * NU - 1;
    static constexpr int ch(int sh) { return sh / 2 - 2 * NU - 1; }
};
constexpr int MG_THREADS = 32 * MG_NW;
static_assert(MG_SH % 4 == 0 && MG_NW <= 32, "tile height");
constexpr int MG_CCW = MG_SW / 2 + 1;      // coarse window of mg_up: 33 columns
constexpr unsigned MG_FULL = 0xffffffffu;

// Window shape of the tiled kernels by window height SH (the width is always
// 64): SH / 4 warps, CH coarse vertices per tile in y, and blocks per SM for
// SCE_TILE_WARPS_PER_SM resident warps (40: a thread keeps 48 registers,
// each of the four schedulers of an SM having 16384; 48: 40 registers, a few
// dozen bytes spilled; twice fewer blocks in FP64).  The solver picks SH per
// grid size (table set by darcy_autotune_tiles; MG_SH otherwise).
template <int SH>
struct MGTile {
    static_assert(SH % 4 == 0 && SH >= 16 && SH <= 64, "tile height");
    static constexpr int H = SH, NW = SH / 4, THREADS = 32 * NW;
    static constexpr int CCH = SH / 2;   // coarse rows of mg_up's window (+ a zero row)
    static constexpr int BPS = SCE_TILE_WARPS_PER_SM / NW;
};

// shared-memory values per block for the 1/diag slices of NW warps (eight
// per thread, see TileBlock)
constexpr int tile_inv_slots(int nw) { return nw * 8 * 32; }

// shared memory: z of rows 0 and 3 of every warp (2 buffers), one row per
// warp for cy / residual exchange, the coarse window of mg_up with a spare row,
// the threads' 1/diag slices
template <typename T, int SH = MG_SH>
constexpr size_t mg_tile_smem_bytes() {
    using G = MGTile<SH>;
    return sizeof(T) * (2 * 2 * G::NW * (size_t)MG_SW + G::NW * (size_t)MG_SW +
                        (size_t)(G::CCH + 1) * MG_CCW + 1 + tile_inv_slots(G::NW));
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
template <> __device__ __forceinline__ float recip<float>(float d) { return __fdividef(1.0f, d); }
template <> __device__ __forceinline__ double recip<double>(double d) { return 1.0 / d; }

// A lane's 2 x 4 block: element e = 2 r + c is window element
// (2 lane + c, 4 warp + r).  Conductances: cxe = cx at the element (edge to
// the east), cyn = cy (edge to the north); cxw0[r] = west edge of the c = 0
// column (from lane - 1), cys0[c] = south edge of row 0 (from warp - 1).
// inv: the lane's 1/diag values in shared memory (element e at inv[32 e]),
// written once by tile_diag and read back by the half-sweeps: each element
// uses its 1/diag once per sweep of its colour, and keeping the eight values in
// registers spilled, so they live in a per-thread slice of shared memory
// (element-major across the lanes, so the accesses are free of bank
// conflicts; only the owning thread reads them, so no barrier is needed).
template <typename T>
struct TileBlock {
    T b[8], z[8], cxe[8], cyn[8], cxw0[4], cys0[2];
    T zs[2], zn[2];   // z of the rows below (r = -1) and above (r = 4) the strip
    T *inv;
};

// 1/diag of element (c, r); c and r are compile-time constants after unrolling
template <typename T>
__device__ __forceinline__ T tile_inv(const TileBlock<T> &t, int c, int r) {
    return t.inv[32 * (2 * r + c)];
}

// Loads b, cx, cy of the block (zero outside the grid); returns the bitmask
// of elements that are unknowns (1 <= gi <= n-1, 0 <= gj <= n).  inside: the
// whole window lies in the grid (block-uniform), so no element needs a bounds
// test and the rows are constant offsets from one base per lane.
template <typename T>
__device__ __forceinline__ unsigned tile_load(TileBlock<T> &t, const T *bs, const T *xs,
                                              const T *ys, int gi0, int gj0, int n,
                                              bool inside) {
    const int w = n + 1;
    unsigned unk = 0;
    if (inside) {
        const long long base = (long long)gj0 * w + gi0;
        const T *pb = bs + base, *px = xs + base, *py = ys + base;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int e = 2 * r + c, o = r * w + c;
                t.b[e] = pb[o];
                t.cxe[e] = px[o];
                t.cyn[e] = py[o];
                if (gi0 + c >= 1 && gi0 + c <= n - 1) unk |= 1u << e;
            }
        }
        return unk;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int e = 2 * r + c, gi = gi0 + c, gj = gj0 + r;
            const bool in = gi >= 0 && gi <= n && gj >= 0 && gj <= n;
            const long long g = (long long)gj * w + gi;
            t.b[e] = in ? bs[g] : T(0);
            t.cxe[e] = in ? xs[g] : T(0);
            t.cyn[e] = in ? ys[g] : T(0);
            if (in && gi >= 1 && gi <= n - 1) unk |= 1u << e;
        }
    }
    return unk;
}

// West/south edge conductances from the neighbouring lane / warp (xrow: one
// shared row per warp), then 1/diag of the lane's elements (0 where not an
// unknown: Dirichlet column, outside the grid, so their z stays 0) into its
// slice of sinv (tile_inv_slots(NW) values).  Contains a barrier.  NW: warps
// of the block.
template <typename T, int NW = MG_NW>
__device__ __forceinline__ void tile_diag(TileBlock<T> &t, T *xrow, int lane, int warp,
                                          unsigned unk, T *sinv) {
#pragma unroll
    for (int r = 0; r < 4; ++r) t.cxw0[r] = __shfl_up_sync(MG_FULL, t.cxe[2 * r + 1], 1);
    xrow[warp * MG_SW + 2 * lane] = t.cyn[6];
    xrow[warp * MG_SW + 2 * lane + 1] = t.cyn[7];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 2; ++c)
        t.cys0[c] = warp > 0 ? xrow[(warp - 1) * MG_SW + 2 * lane + c] : T(0);
    t.inv = sinv + warp * 8 * 32 + lane;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int e = 2 * r + c;
            const T cw = c == 0 ? t.cxw0[r] : t.cxe[2 * r];
            const T cs = r == 0 ? t.cys0[c] : t.cyn[2 * (r - 1) + c];
            t.inv[32 * e] = ((unk >> e) & 1) ? recip(cw + t.cxe[e] + cs + t.cyn[e]) : T(0);
        }
    }
}

// Publishes rows 0 and 3 of z in buffer buf, waits, and reads the rows below
// and above the strip (zero beyond the window).  NW: warps of the block.
template <typename T, int NW = MG_NW>
__device__ __forceinline__ void tile_exchange(TileBlock<T> &t, T *xz, int buf, int lane,
                                              int warp) {
    T *lo = xz + (buf * 2 + 0) * NW * MG_SW, *hi = xz + (buf * 2 + 1) * NW * MG_SW;
    lo[warp * MG_SW + 2 * lane] = t.z[0];
    lo[warp * MG_SW + 2 * lane + 1] = t.z[1];
    hi[warp * MG_SW + 2 * lane] = t.z[6];
    hi[warp * MG_SW + 2 * lane + 1] = t.z[7];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        t.zs[c] = warp > 0 ? hi[(warp - 1) * MG_SW + 2 * lane + c] : T(0);
        t.zn[c] = warp < NW - 1 ? lo[(warp + 1) * MG_SW + 2 * lane + c] : T(0);
    }
}

// Neighbours of element (c, r) in the order west, east, south, north: their z
// and the conductances of the four edges.  The horizontal neighbour in the
// next lane comes by shuffle, so every lane of the warp must call this for
// the same (c, r).  EAST0: the window's last column is the grid's last
// unknown column, whose east neighbour (the Dirichlet column) has z = 0.
template <typename T, int C, int R, bool EAST0 = false>
__device__ __forceinline__ void tile_nbrs(const TileBlock<T> &t, T *zw, T *ze, T *zsv, T *znv,
                                          T *cw, T *cs) {
    if constexpr (C == 0) {
        *zw = __shfl_up_sync(MG_FULL, t.z[2 * R + 1], 1);
        *ze = t.z[2 * R + 1];
        *cw = t.cxw0[R];
    } else {
        *zw = t.z[2 * R];
        *ze = __shfl_down_sync(MG_FULL, t.z[2 * R], 1);
        if constexpr (EAST0) {
            if ((threadIdx.x & 31) == 31) *ze = T(0);
        }
        *cw = t.cxe[2 * R];
    }
    *zsv = R == 0 ? t.zs[C] : t.z[2 * (R - 1) + C];
    *znv = R == 3 ? t.zn[C] : t.z[2 * (R + 1) + C];
    *cs = R == 0 ? t.cys0[C] : t.cyn[2 * (R - 1) + C];
}

// One Gauss-Seidel half-sweep over the elements of colour COL of the block.
template <typename T, int COL, int R = 0, bool EAST0 = false>
__device__ __forceinline__ void tile_half_sweep(TileBlock<T> &t) {
    if constexpr (R < 4) {
        constexpr int C = (COL + R) & 1, e = 2 * R + C;
        T zw, ze, zsv, znv, cw, cs;
        tile_nbrs<T, C, R, EAST0>(t, &zw, &ze, &zsv, &znv, &cw, &cs);
        t.z[e] = (t.b[e] + cw * zw + t.cxe[e] * ze + cs * zsv + t.cyn[e] * znv) * tile_inv(t, C, R);
        tile_half_sweep<T, COL, R + 1, EAST0>(t);
    }
}

// Residual b - A z at the red element of row R (c = R % 2); 0 where not an unknown.
template <typename T, int R, bool EAST0 = false>
__device__ __forceinline__ T tile_red_residual(const TileBlock<T> &t, unsigned unk) {
    constexpr int C = R & 1, e = 2 * R + C;
    T zw, ze, zsv, znv, cw, cs;
    tile_nbrs<T, C, R, EAST0>(t, &zw, &ze, &zsv, &znv, &cw, &cs);
    const T zc = t.z[e];
    const T rv = t.b[e] - (cw * (zc - zw) + t.cxe[e] * (zc - ze) + cs * (zc - zsv) +
                           t.cyn[e] * (zc - znv));
    return ((unk >> e) & 1) ? rv : T(0);
}

template <typename T, int SH = MG_SH, int NU = mg_nu<T>()>
__global__ void __launch_bounds__(MGTile<SH>::THREADS, sizeof(T) == 4 ? MGTile<SH>::BPS : MGTile<SH>::BPS / 2) mg_down_kernel(
    const T *__restrict__ cx, const T *__restrict__ cy, const T *__restrict__ b,
    T *__restrict__ zpre, int n, T *__restrict__ bc, int tiles_x, const int *__restrict__ act) {
    using G = MGTile<SH>;
    using GM = MGGeom<T, NU>;
    constexpr int MG_SH = SH, MG_NW = G::NW, MG_CH = GM::ch(SH), MG_CW = GM::CW, MG_OD = GM::OD;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xz = reinterpret_cast<T *>(smem_raw);
    T *xrow = xz + 2 * 2 * MG_NW * MG_SW;
    T *sinv = xrow + MG_NW * MG_SW;
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nc = n / 2, w = n + 1, wc = nc + 1;
    const long long V = (long long)w * w, Vc = (long long)wc * wc;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int I0 = tx * MG_CW, J0 = ty * MG_CH;
    const int gi0 = 2 * I0 - MG_OD + 2 * lane, gj0 = 2 * J0 - MG_OD + 4 * warp;
    const bool inside = 2 * I0 - MG_OD >= 0 && 2 * I0 - MG_OD + MG_SW - 1 <= n &&
                        2 * J0 - MG_OD >= 0 && 2 * J0 - MG_OD + MG_SH - 1 <= n;
    TileBlock<T> t;
    const unsigned unk = tile_load(t, b + s * V, cx + s * V, cy + s * V, gi0, gj0, n, inside);
    tile_diag<T, MG_NW>(t, xrow, lane, warp, unk, sinv);
    // red from z = 0: z = b / diag at red elements ((c + r) even), 0 at black
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int e = 2 * r + c;
            t.z[e] = ((c + r) & 1) == 0 ? t.b[e] * tile_inv(t, c, r) : T(0);
        }
    }
    tile_exchange<T, MG_NW>(t, xz, 0, lane, warp);
    tile_half_sweep<T, 1>(t);
    tile_exchange<T, MG_NW>(t, xz, 1, lane, warp);
#pragma unroll
    for (int k = 1; k < NU; ++k) {   // the further sweeps: red, black
        tile_half_sweep<T, 0>(t);
        tile_exchange<T, MG_NW>(t, xz, 0, lane, warp);
        tile_half_sweep<T, 1>(t);
        tile_exchange<T, MG_NW>(t, xz, 1, lane, warp);
    }
    // red residuals of rows 0..3 (c = r % 2)
    const T r0 = tile_red_residual<T, 0>(t, unk), r1 = tile_red_residual<T, 1>(t, unk);
    const T r2 = tile_red_residual<T, 2>(t, unk), r3 = tile_red_residual<T, 3>(t, unk);
    // row 3's red residual (c = 1) to the warp above, for its row -1
    xrow[warp * MG_SW + lane] = r3;
    __syncthreads();
    const T rm = warp > 0 ? xrow[(warp - 1) * MG_SW + lane] : T(0);
    const T l1 = __shfl_up_sync(MG_FULL, r1, 1), l3 = __shfl_up_sync(MG_FULL, r3, 1);
    const T lm = __shfl_up_sync(MG_FULL, rm, 1);
    // coarse vertices at (c = 0, r = 0) and (c = 0, r = 2): centre + 1/4 x the
    // four diagonal (red) neighbours, in the order SW, SE, NW, NE
    const int I = I0 - MG_OD / 2 + lane, Jb = J0 - MG_OD / 2 + 2 * warp;
    const T acc[2] = {T(0.25) * (lm + rm + l1 + r1) + r0, T(0.25) * (l1 + r1 + l3 + r3) + r2};
    T *bcs = bc + s * Vc;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int J = Jb + k;
        if (I - I0 >= 0 && I - I0 < MG_CW && J - J0 >= 0 && J - J0 < MG_CH && I <= nc && J <= nc)
            bcs[(long long)J * wc + I] = (I > 0 && I < nc) ? acc[k] : T(0);
    }
    // owned fine vertices: window [OD, OD + 2 CW) x [OD, OD + 2 CH)
    T *zs = zpre + s * V;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int li = 2 * lane + c, lj = 4 * warp + r;
            const int gi = gi0 + c, gj = gj0 + r;
            if (li >= MG_OD && li < MG_OD + 2 * MG_CW && lj >= MG_OD &&
                lj < MG_OD + 2 * MG_CH && gi <= n && gj <= n)
                zs[(long long)gj * w + gi] = t.z[2 * r + c];
        }
    }
}

template <typename T, int SH = MG_SH, int NU = mg_nu<T>()>
__global__ void __launch_bounds__(MGTile<SH>::THREADS, sizeof(T) == 4 ? MGTile<SH>::BPS : MGTile<SH>::BPS / 2) mg_up_kernel(
    const T *__restrict__ cx, const T *__restrict__ cy, const T *__restrict__ b,
    const T *__restrict__ zpre, T *__restrict__ z, int n, const T *__restrict__ zc, int tiles_x,
    const int *__restrict__ act, double *__restrict__ part_rz, int nblk) {
    using G = MGTile<SH>;
    using GM = MGGeom<T, NU>;
    constexpr int MG_SH = SH, MG_NW = G::NW, MG_CH = GM::ch(SH), MG_CCH = G::CCH;
    constexpr int MG_CW = GM::CW, MG_OU = GM::OU;
    constexpr int MG_THREADS = G::THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T sred[32];
    T *xz = reinterpret_cast<T *>(smem_raw);
    T *xrow = xz + 2 * 2 * MG_NW * MG_SW;
    T *szc = xrow + MG_NW * MG_SW;   // coarse window, row stride MG_CCW, MG_CCH + 1 rows
    T *sinv = szc + (MG_CCH + 1) * MG_CCW + 1;
    const int s = blockIdx.y;
    if (!act[s]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nc = n / 2, w = n + 1, wc = nc + 1;
    const long long V = (long long)w * w, Vc = (long long)wc * wc;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int I0 = tx * MG_CW, J0 = ty * MG_CH;
    const int gi0 = 2 * I0 - MG_OU + 2 * lane, gj0 = 2 * J0 - MG_OU + 4 * warp;
    const int cox = I0 - MG_OU / 2, coy = J0 - MG_OU / 2;
    const T *zcs = zc + s * Vc;
    for (int q = threadIdx.x; q < (MG_CCH + 1) * MG_CCW + 1; q += MG_THREADS) {
        const int ci = q % MG_CCW, cj = q / MG_CCW;
        const int I = cox + ci, J = coy + cj;
        szc[q] = (cj < MG_CCH && I >= 0 && I <= nc && J >= 0 && J <= nc)
                     ? zcs[(long long)J * wc + I] : T(0);
    }
    const bool inside = 2 * I0 - MG_OU >= 0 && 2 * I0 - MG_OU + MG_SW - 1 <= n &&
                        2 * J0 - MG_OU >= 0 && 2 * J0 - MG_OU + MG_SH - 1 <= n;
    TileBlock<T> t;
    const unsigned unk = tile_load(t, b + s * V, cx + s * V, cy + s * V, gi0, gj0, n, inside);
    const T *zps = zpre + s * V;
    if (inside) {
        const T *pz = zps + (long long)gj0 * w + gi0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) t.z[2 * r + c] = pz[r * w + c];
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int gi = gi0 + c, gj = gj0 + r;
                t.z[2 * r + c] = (gi >= 0 && gi <= n && gj >= 0 && gj <= n)
                                     ? zps[(long long)gj * w + gi] : T(0);
            }
        }
    }
    tile_diag<T, MG_NW>(t, xrow, lane, warp, unk, sinv);   // its barrier also covers szc
    // z += P zc: coarse column lane (and lane + 1), rows 2 warp + {0, 1, 2};
    // weights (1, 0) at even fine indices, (1/2, 1/2) at odd ones
    const T *q0 = szc + (2 * warp) * MG_CCW + lane;
    const T a0 = q0[0], a1 = q0[1], b0 = q0[MG_CCW], b1 = q0[MG_CCW + 1];
    const T c0 = q0[2 * MG_CCW], c1 = q0[2 * MG_CCW + 1];
    const T h = T(0.5), qq = T(0.25);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!((unk >> k) & 1)) continue;
        const int r = k >> 1, c = k & 1;
        T pv;
        const T x0 = r < 2 ? a0 : b0, x1 = r < 2 ? a1 : b1;   // row J_lo
        const T y0 = r < 2 ? b0 : c0, y1 = r < 2 ? b1 : c1;   // row J_lo + 1
        if ((r & 1) == 0) pv = c == 0 ? x0 : h * (x0 + x1);
        else pv = c == 0 ? h * (x0 + y0) : qq * ((x0 + x1) + (y0 + y1));
        t.z[k] += pv;
    }
    tile_exchange<T, MG_NW>(t, xz, 0, lane, warp);
    tile_half_sweep<T, 1>(t);
    tile_exchange<T, MG_NW>(t, xz, 1, lane, warp);
    tile_half_sweep<T, 0>(t);
#pragma unroll
    for (int k = 1; k < NU; ++k) {   // the further sweeps: black, red
        tile_exchange<T, MG_NW>(t, xz, 0, lane, warp);
        tile_half_sweep<T, 1>(t);
        tile_exchange<T, MG_NW>(t, xz, 1, lane, warp);
        tile_half_sweep<T, 0>(t);
    }
    // owned fine vertices: window [OU, OU + 2 CW) x [OU, OU + 2 CH)
    T *zs = z + s * V;
    T rz = T(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int li = 2 * lane + c, lj = 4 * warp + r;
            const int gi = gi0 + c, gj = gj0 + r;
            if (li >= MG_OU && li < MG_OU + 2 * MG_CW && lj >= MG_OU &&
                lj < MG_OU + 2 * MG_CH && gi <= n && gj <= n) {
                zs[(long long)gj * w + gi] = t.z[2 * r + c];
                rz += t.b[2 * r + c] * t.z[2 * r + c];
            }
        }
    }
    if (part_rz) {
        const T tot = block_sum_t(rz, sred);
        if (threadIdx.x == 0) part_rz[(long long)s * nblk + blockIdx.x] = (double)tot;
    }
}

struct TailPtrs {
    void *cx[8], *cy[8];
};

// V-cycle of levels NT_N, NT_N/2, ..., 2 of one sample per block: nu0 sweeps
// per side on level NT_N, nuc on the levels below.
template <typename T, int NT_N, int NTHR>
__global__ void __launch_bounds__(NTHR) mg_tail_kernel(TailPtrs tp, const T *__restrict__ b,
                                                       T *__restrict__ z,
                                                       const int *__restrict__ act,
                                                       double *__restrict__ part_rz, int nu0,
                                                       int nuc) {
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
    block_vcycle<T, NT_N, NTHR, Lay>(base, nu0, nuc);
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

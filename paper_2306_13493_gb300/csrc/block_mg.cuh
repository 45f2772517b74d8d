// Multigrid V(nu, nu) cycle executed by one thread block on one sample whose
// level arrays are in shared memory (levels N, N/2, ..., 2).  Shared by the
// one-block-per-sample solver and by the coarse-level tail of the batched
// solver.  Level sizes and array offsets are compile-time constants (the
// level recursion is unrolled; arrays are addressed as base + constant), and
// each Gauss-Seidel half-sweep visits only the vertices of its colour.
#pragma once

#include "stencil.cuh"

namespace sce {

constexpr int mg_levels(int n) { return n <= 2 ? 1 : 1 + mg_levels(n / 2); }

// Red-black Gauss-Seidel sweeps before and after each coarse-grid correction
// on the finest level of the batched FP32 solver's cycle and on its levels
// wider than 128 cells (the coarser levels take three by default):
// SCE_MG_NU = 2 (the default: ~27 % fewer CG iterations than one sweep for
// ~1.3-1.45 times the work of a cycle), or 1.
#ifndef SCE_MG_NU
#define SCE_MG_NU 2
#endif
constexpr int MG_NU = SCE_MG_NU;
static_assert(MG_NU == 1 || MG_NU == 2, "sweeps per side of the cycle");

// Sweeps per side for element type T: the FP32 path takes MG_NU; the FP64
// path keeps V(1,1), since its smoothing runs on GB300's FP64 pipe (~1/64 of
// the FP32 rate), where V(2,2) measured 10 % slower over a whole sweep.
template <typename T>
constexpr int mg_nu() {
    return sizeof(T) == 4 ? MG_NU : 1;
}

// Barrier of an NT-thread block: a single-warp block (NT == 32) only needs
// the warp's own synchronisation, which also orders its shared-memory
// accesses.
template <int NT>
__device__ __forceinline__ void block_sync() {
    if constexpr (NT == 32) __syncwarp();
    else __syncthreads();
}
constexpr int mg_vof(int n) { return (n + 1) * (n + 1); }

// Row pitch of a level of n cells in a shared-memory hierarchy: n + 1, or
// n + 2 with PAD on the levels of at least 32 cells.  With the odd pitch n + 1
// every vertex of one colour sits at an address of one parity, so a warp's
// red-black half-sweep reaches only half of the 32 banks (two accesses per
// bank); the even pitch alternates the parity from row to row, and the rows
// of one colour a warp covers fill all the banks.
constexpr int mg_pitch(int n, bool pad) { return n + 1 + ((pad && n >= 32) ? 1 : 0); }

// Array k (0 cx, 1 cy, 2 b, 3 z) of level L of an N-cell hierarchy, all levels
// stored one after the other, each as [cx | cy | b | z], rows of pitch(L)
// values (the padding column is never read).
template <int N, bool PAD = false> struct MGPackedLayout {
    static constexpr int pitch(int L) { return mg_pitch(N >> L, PAD); }
    static constexpr int size(int L) { return ((N >> L) + 1) * pitch(L); }
    static constexpr int off(int L, int k) {
        int o = 0;
        for (int l = 0; l < L; ++l) o += 4 * size(l);
        return o + k * size(L);
    }
    static constexpr int total() { return off(mg_levels(N), 0); }
};

// One red-black half-sweep of colour c on level nL (row pitch PW): vertex
// (i, j) with (i + j) % 2 == c, 1 <= i <= nL-1.
template <typename T, int nL, int NT, int PW = nL + 1>
__device__ __forceinline__ void block_half_sweep(const T *cx, const T *cy, const T *b, T *z,
                                                 int c) {
    constexpr int W = nL + 1;
    constexpr int HW = (nL + 2) / 2;   // colour vertices per row (upper bound)
    for (int k = threadIdx.x; k < W * HW; k += NT) {
        const int j = k / HW;
        const int i = 2 * (k - j * HW) + ((j + c) & 1);
        if (i >= 1 && i <= nL - 1) smooth_at(cx, cy, b, z, i, j, nL, PW);
    }
}

template <typename T, int N, int NT, class Lay, int L, int WARP_N, int NU>
__device__ __forceinline__ void block_vcycle_level(T *base, int nu0, int nuc);

// The V-cycle from level L down and back up: with WARP_N > 0 in a block of
// more than one warp, the levels of at most WARP_N cells run on warp 0 alone
// (warp synchronisation) while the other warps wait at one block barrier.
// nu0: sweeps per side on level 0, nuc on the others (compile-time constants
// where the caller passes them so, and the sweep loops unroll).
template <typename T, int N, int NT, class Lay, int L, int WARP_N, int NU>
__device__ __forceinline__ void block_vcycle_from(T *base, int nu0, int nuc) {
    if constexpr (NT > 32 && WARP_N > 0 && (N >> L) <= WARP_N) {
        if (threadIdx.x < 32) block_vcycle_level<T, N, 32, Lay, L, 0, NU>(base, nu0, nuc);
        __syncthreads();
    } else {
        block_vcycle_level<T, N, NT, Lay, L, WARP_N, NU>(base, nu0, nuc);
    }
}

template <typename T, int N, int NT, class Lay, int L, int WARP_N, int NU>
__device__ __forceinline__ void block_vcycle_level(T *base, int nu0, int nuc) {
    constexpr int NL = mg_levels(N);
    constexpr int nL = N >> L;
    T *cx = base + Lay::off(L, 0), *cy = base + Lay::off(L, 1);
    T *b = base + Lay::off(L, 2), *z = base + Lay::off(L, 3);
    if constexpr (L == NL - 1) {
        static_assert(Lay::pitch(L) == 3, "the coarsest level is dense");
        if (threadIdx.x == 0) coarsest_solve(cx, cy, b, z);
        block_sync<NT>();
    } else {
        constexpr int nc = nL / 2, wc = nc + 1, Vc = wc * wc, wL = nL + 1, VL = wL * wL;
        constexpr int PL = Lay::pitch(L), PC = Lay::pitch(L + 1);
        T *bc = base + Lay::off(L + 1, 2), *zc = base + Lay::off(L + 1, 3);
        const int nu = L == 0 ? nu0 : nuc;
#pragma unroll
        for (int k = 0; k < nu; ++k) {
            block_half_sweep<T, nL, NT, PL>(cx, cy, b, z, 0);
            block_sync<NT>();
            block_half_sweep<T, nL, NT, PL>(cx, cy, b, z, 1);
            block_sync<NT>();
        }
        for (int v = threadIdx.x; v < Vc; v += NT) {
            const int J = v / wc, I = v - J * wc, q = J * PC + I;
            bc[q] = (I > 0 && I < nc) ? restrict_at(cx, cy, b, z, nL, I, J, PL) : T(0);
            zc[q] = T(0);
        }
        block_sync<NT>();
        block_vcycle_from<T, N, NT, Lay, L + 1, WARP_N, NU>(base, nu0, nuc);
        for (int v = threadIdx.x; v < VL; v += NT) {
            const int j = v / wL, i = v - j * wL;
            if (i > 0 && i < nL) z[j * PL + i] += prolong_at(zc, nc, i, j, PC);
        }
        block_sync<NT>();
#pragma unroll
        for (int k = 0; k < nu; ++k) {
            block_half_sweep<T, nL, NT, PL>(cx, cy, b, z, 1);
            block_sync<NT>();
            block_half_sweep<T, nL, NT, PL>(cx, cy, b, z, 0);
            block_sync<NT>();
        }
    }
}

// Coarse conductances of levels L..NL-1 from level L-1 (call with L = 1).
template <typename T, int N, int NT, class Lay, int L>
__device__ __forceinline__ void block_coarsen(T *base) {
    if constexpr (L < mg_levels(N)) {
        constexpr int nL = N >> L, wL = nL + 1, VL = wL * wL;
        constexpr int PF = Lay::pitch(L - 1), PL = Lay::pitch(L);
        const T *fx = base + Lay::off(L - 1, 0), *fy = base + Lay::off(L - 1, 1);
        T *cx = base + Lay::off(L, 0), *cy = base + Lay::off(L, 1);
        for (int v = threadIdx.x; v < VL; v += NT) {
            const int J = v / wL, I = v - J * wL;
            T gx, gy;
            coarsen_at(fx, fy, 2 * nL, I, J, &gx, &gy, PF);
            cx[J * PL + I] = gx;
            cy[J * PL + I] = gy;
        }
        block_sync<NT>();
        block_coarsen<T, N, NT, Lay, L + 1>(base);
    }
}

// z = M^{-1} b on level 0 of the hierarchy laid out by Lay from `base`.
// Symmetric: on each level, nu red-black Gauss-Seidel sweeps before the
// restriction and nu black-red sweeps after the prolongation (nu = nu0 on
// level 0, nuc below it; both NU by default), exact solve on 2 cells.  All NT
// threads must call it.
template <typename T, int N, int NT, class Lay, int WARP_N = 0, int NU = mg_nu<T>()>
__device__ __forceinline__ void block_vcycle(T *base, int nu0 = NU, int nuc = NU) {
    T *z = base + Lay::off(0, 3);
    for (int v = threadIdx.x; v < Lay::size(0); v += NT) z[v] = T(0);
    block_sync<NT>();
    block_vcycle_from<T, N, NT, Lay, 0, WARP_N, NU>(base, nu0, nuc);
}

}  // namespace sce

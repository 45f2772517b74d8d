// Multigrid V(1,1) cycle executed by one thread block on one sample whose
// level arrays are in shared memory (levels N, N/2, ..., 2).  Shared by the
// one-block-per-sample solver and by the coarse-level tail of the batched
// solver.
#pragma once

#include "stencil.cuh"

namespace sce {

// z[0] = M^{-1} b[0] for the hierarchy (cx[L], cy[L], bb[L], zz[L]), L < NL,
// level L having N >> L cells.  Symmetric: red-black Gauss-Seidel before the
// restriction, black-red after the prolongation, exact solve on 2 cells.
// All NT threads of the block must call it.
template <typename T, int N, int NT>
__device__ __forceinline__ void block_vcycle(T *const *cx, T *const *cy, T *const *bb, T *const *zz,
                                             int NL) {
    const int tid = threadIdx.x;
    {
        const int V = (N + 1) * (N + 1);
        for (int v = tid; v < V; v += NT) zz[0][v] = T(0);
    }
    __syncthreads();
    for (int L = 0; L < NL - 1; ++L) {
        const int nL = N >> L, wL = nL + 1, VL = wL * wL;
        for (int c = 0; c < 2; ++c) {
            for (int v = tid; v < VL; v += NT) {
                const int j = v / wL, i = v - j * wL;
                if (i > 0 && i < nL && ((i + j) & 1) == c) smooth_at(cx[L], cy[L], bb[L], zz[L], i, j, nL);
            }
            __syncthreads();
        }
        const int nc = nL / 2, wc = nc + 1, Vc = wc * wc;
        for (int v = tid; v < Vc; v += NT) {
            const int J = v / wc, I = v - J * wc;
            bb[L + 1][v] = (I > 0 && I < nc) ? restrict_at(cx[L], cy[L], bb[L], zz[L], nL, I, J) : T(0);
            zz[L + 1][v] = T(0);
        }
        __syncthreads();
    }
    if (tid == 0) coarsest_solve(cx[NL - 1], cy[NL - 1], bb[NL - 1], zz[NL - 1]);
    __syncthreads();
    for (int L = NL - 2; L >= 0; --L) {
        const int nL = N >> L, wL = nL + 1, VL = wL * wL;
        for (int v = tid; v < VL; v += NT) {
            const int j = v / wL, i = v - j * wL;
            if (i > 0 && i < nL) zz[L][v] += prolong_at(zz[L + 1], nL / 2, i, j);
        }
        __syncthreads();
        for (int c = 1; c >= 0; --c) {
            for (int v = tid; v < VL; v += NT) {
                const int j = v / wL, i = v - j * wL;
                if (i > 0 && i < nL && ((i + j) & 1) == c) smooth_at(cx[L], cy[L], bb[L], zz[L], i, j, nL);
            }
            __syncthreads();
        }
    }
}

}  // namespace sce

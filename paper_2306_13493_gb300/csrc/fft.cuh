// Shared-memory FFT of one line of length N = 2^logN with the +i exponent of
// the paper's Fourier matrix (Eq. (2.6)), unnormalised:
//     X[p] = sum_q x[q] exp(+2 pi i p q / N).
// Stockham autosort formulation (radix-4 stages, one radix-2 stage when logN
// is odd): stage with span Ns reads x[j + r N/R], r < R, twiddles input r by
// W^(r (j mod Ns) N/(R Ns)), W = exp(2 pi i / N), applies the R-point DFT and
// writes y[(j div Ns) R Ns + (j mod Ns) + r Ns].  Each thread keeps its
// butterflies' inputs in registers across a barrier, so the stage runs in
// place in one shared buffer.
#pragma once

namespace sce {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R2> __device__ __forceinline__ R2 cadd(R2 a, R2 b) { return {a.x + b.x, a.y + b.y}; }
template <typename R2> __device__ __forceinline__ R2 csub(R2 a, R2 b) { return {a.x - b.x, a.y - b.y}; }
template <typename R2> __device__ __forceinline__ R2 cmul(R2 a, R2 b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// i * a
template <typename R2> __device__ __forceinline__ R2 cmuli(R2 a) { return {-a.y, a.x}; }

// Shared-memory line layout: element i of a line lives at fft_pad(i), one
// padding slot per 16 complex values, so the strided writes of the first
// Stockham stages (stride 4 and 16 elements) hit distinct banks.
__host__ __device__ constexpr int fft_pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int fft_line_pitch(int P) { return P + (P >> 4); }

// MAXB = maximum butterflies per thread per stage (N/4 <= MAXB * nthr).
// buf is a padded line (fft_pad indexing).
template <typename R, int MAXB>
__device__ __forceinline__ void smem_fft(typename C2<R>::T *buf, int logN,
                                         const typename C2<R>::T *__restrict__ tw, int tid,
                                         int nthr) {
    using R2 = typename C2<R>::T;
    const int N = 1 << logN;
    int Ns = 1;
    const int nb4 = N >> 2;
    for (; (Ns << 2) <= N; Ns <<= 2) {
        R2 v[MAXB][4];
        int jj[MAXB];
#pragma unroll
        for (int b = 0; b < MAXB; ++b) {
            const int j = tid + b * nthr;
            jj[b] = j;
            if (j < nb4) {
#pragma unroll
                for (int r = 0; r < 4; ++r) v[b][r] = buf[fft_pad(j + r * nb4)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < MAXB; ++b) {
            const int j = jj[b];
            if (j < nb4) {
                const int k = j & (Ns - 1);
                if (Ns > 1) {
                    const int step = k * (N / (4 * Ns));
                    v[b][1] = cmul(v[b][1], tw[step]);
                    v[b][2] = cmul(v[b][2], tw[2 * step]);
                    v[b][3] = cmul(v[b][3], tw[3 * step]);
                }
                const R2 a02 = cadd(v[b][0], v[b][2]);
                const R2 s02 = csub(v[b][0], v[b][2]);
                const R2 a13 = cadd(v[b][1], v[b][3]);
                const R2 s13 = cmuli(csub(v[b][1], v[b][3]));
                const int o = (j - k) * 4 + k;
                buf[fft_pad(o)] = cadd(a02, a13);
                buf[fft_pad(o + Ns)] = cadd(s02, s13);
                buf[fft_pad(o + 2 * Ns)] = csub(a02, a13);
                buf[fft_pad(o + 3 * Ns)] = csub(s02, s13);
            }
        }
        __syncthreads();
    }
    if (Ns < N) {   // one radix-2 stage, Ns = N/2
        const int nb2 = N >> 1;
        R2 v[2 * MAXB][2];
#pragma unroll
        for (int b = 0; b < 2 * MAXB; ++b) {
            const int j = tid + b * nthr;
            if (j < nb2) {
                v[b][0] = buf[fft_pad(j)];
                v[b][1] = buf[fft_pad(j + nb2)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < 2 * MAXB; ++b) {
            const int j = tid + b * nthr;
            if (j < nb2) {
                const R2 t = (Ns > 1) ? cmul(v[b][1], tw[j]) : v[b][1];   // k = j, step = 1
                buf[fft_pad(j)] = cadd(v[b][0], t);
                buf[fft_pad(j + Ns)] = csub(v[b][0], t);
            }
        }
        __syncthreads();
    }
}

}  // namespace sce

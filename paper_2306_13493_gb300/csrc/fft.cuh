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

// ---------------------------------------------------------------- radix 16
// The same transform with radix-16 Stockham passes (a final radix-2/4/8 pass
// when logN is not a multiple of 4): each thread holds the 16 inputs of one
// butterfly in registers, so a 2048-point line takes 3 shared-memory rounds
// instead of 6.  Requires exactly 16 elements per thread (nthr = N/16).  The
// 16-point DFT is two layers of 4-point DFTs with the twiddles w16^(p1 q2)
// between them (16 = 4 x 4: q = 4 q1 + q2, p = p1 + 4 p2).

// 4-point DFT with the +i exponent, in place (outputs in natural order)
template <typename R2>
__device__ __forceinline__ void dft4(R2 &x0, R2 &x1, R2 &x2, R2 &x3) {
    const R2 a02 = cadd(x0, x2), s02 = csub(x0, x2);
    const R2 a13 = cadd(x1, x3), s13 = cmuli(csub(x1, x3));
    x0 = cadd(a02, a13);
    x1 = cadd(s02, s13);
    x2 = csub(a02, a13);
    x3 = csub(s02, s13);
}

// (x + iy) (c + is)
template <typename R2, typename R>
__device__ __forceinline__ R2 cmulc(R2 a, R c, R s) {
    return {a.x * c - a.y * s, a.x * s + a.y * c};
}

// v *= exp(2 pi i m / 16) for the exponents m = p1 q2 of the 16-point DFT
template <typename R2, typename R>
__device__ __forceinline__ R2 w16(R2 v, int m) {
    const R c1 = R(0.923879532511286756128), s1 = R(0.382683432365089771728);
    const R h = R(0.707106781186547524401);
    switch (m) {
        case 1: return cmulc(v, c1, s1);
        case 2: return cmulc(v, h, h);
        case 3: return cmulc(v, s1, c1);
        case 4: return cmuli(v);
        case 6: return cmulc(v, -h, h);
        case 9: return cmulc(v, -c1, -s1);
        default: return v;
    }
}

// 16-point DFT (+i) of v[0..15]; X[p1 + 4 p2] ends in v[4 p1 + p2]
template <typename R2, typename R>
__device__ __forceinline__ void dft16(R2 v[16]) {
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) dft4(v[q2], v[4 + q2], v[8 + q2], v[12 + q2]);
    // v[q2 + 4 p1] = T[q2][p1]; twiddle, then transpose into v[4 p1 + q2]
    R2 t[16];
#pragma unroll
    for (int p1 = 0; p1 < 4; ++p1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) t[4 * p1 + q2] = w16<R2, R>(v[q2 + 4 * p1], p1 * q2);
#pragma unroll
    for (int p1 = 0; p1 < 4; ++p1) dft4(t[4 * p1], t[4 * p1 + 1], t[4 * p1 + 2], t[4 * p1 + 3]);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = t[q];
}

// final pass of radix RF (2, 4, 8): butterfly j reads x[j + r N/RF], writes
// y[j + p Ns] (Ns = N/RF, the last Stockham stage), twiddles tw[r j]
template <typename R2, typename R, int RF>
__device__ __forceinline__ void fft_last_pass(R2 *buf, int N, const R2 *__restrict__ tw,
                                              int tid, int nthr) {
    constexpr int NB = 16 / RF;   // butterflies per thread (16 elements per thread)
    const int Ns = N / RF;
    R2 v[NB][RF];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = tid + b * nthr;
#pragma unroll
        for (int r = 0; r < RF; ++r) v[b][r] = buf[fft_pad(j + r * Ns)];
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = tid + b * nthr;
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RF; ++r) v[b][r] = cmul(v[b][r], tw[r * j]);
        }
        if constexpr (RF == 2) {
            const R2 a = v[b][0];
            v[b][0] = cadd(a, v[b][1]);
            v[b][1] = csub(a, v[b][1]);
        } else if constexpr (RF == 4) {
            dft4(v[b][0], v[b][1], v[b][2], v[b][3]);
        } else {
            // 8 = 4 x 2: DFT4 of the even and odd inputs, odd twiddled by w8^p
            R2 e0 = v[b][0], e1 = v[b][2], e2 = v[b][4], e3 = v[b][6];
            R2 o0 = v[b][1], o1 = v[b][3], o2 = v[b][5], o3 = v[b][7];
            dft4(e0, e1, e2, e3);
            dft4(o0, o1, o2, o3);
            const R h = R(0.707106781186547524401);
            o1 = cmulc(o1, h, h);
            o2 = cmuli(o2);
            o3 = cmulc(o3, -h, h);
            v[b][0] = cadd(e0, o0);
            v[b][4] = csub(e0, o0);
            v[b][1] = cadd(e1, o1);
            v[b][5] = csub(e1, o1);
            v[b][2] = cadd(e2, o2);
            v[b][6] = csub(e2, o2);
            v[b][3] = cadd(e3, o3);
            v[b][7] = csub(e3, o3);
        }
#pragma unroll
        for (int p = 0; p < RF; ++p) buf[fft_pad(j + p * Ns)] = v[b][p];
    }
    __syncthreads();
}

// Passes from span Ns on (Ns = 1: the whole transform).
template <typename R>
__device__ __forceinline__ void smem_fft16_from(typename C2<R>::T *buf, int logN,
                                                const typename C2<R>::T *__restrict__ tw, int tid,
                                                int nthr, int Ns) {
    using R2 = typename C2<R>::T;
    const int N = 1 << logN;
    const int nb16 = N >> 4;   // == nthr
    for (; (Ns << 4) <= N; Ns <<= 4) {
        R2 v[16];
        const int j = tid;
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = buf[fft_pad(j + r * nb16)];
        __syncthreads();
        const int k = j & (Ns - 1);
        if (Ns > 1) {
            const int step = k * (N / (16 * Ns));
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw[r * step]);
        }
        dft16<R2, R>(v);
        const int o = (j - k) * 16 + k;
#pragma unroll
        for (int p = 0; p < 16; ++p) buf[fft_pad(o + p * Ns)] = v[4 * (p & 3) + (p >> 2)];
        __syncthreads();
    }
    const int rf = N / Ns;
    if (rf == 8) fft_last_pass<R2, R, 8>(buf, N, tw, tid, nthr);
    else if (rf == 4) fft_last_pass<R2, R, 4>(buf, N, tw, tid, nthr);
    else if (rf == 2) fft_last_pass<R2, R, 2>(buf, N, tw, tid, nthr);
}

template <typename R>
__device__ __forceinline__ void smem_fft16(typename C2<R>::T *buf, int logN,
                                           const typename C2<R>::T *__restrict__ tw, int tid,
                                           int nthr) {
    smem_fft16_from<R>(buf, logN, tw, tid, nthr, 1);
}

// The radix-16 transform of a line whose first-pass inputs v[r] = x[tid + r N/16]
// are already in registers (loaded by the caller straight from global memory):
// the first pass writes its outputs to the (padded) shared line, the others
// follow.  N >= 16, nthr = N/16.
template <typename R>
__device__ __forceinline__ void smem_fft16_regs(typename C2<R>::T *buf,
                                                typename C2<R>::T v[16], int logN,
                                                const typename C2<R>::T *__restrict__ tw,
                                                int tid, int nthr) {
    dft16<typename C2<R>::T, R>(v);
#pragma unroll
    for (int p = 0; p < 16; ++p) buf[fft_pad(16 * tid + p)] = v[4 * (p & 3) + (p >> 2)];
    __syncthreads();
    smem_fft16_from<R>(buf, logN, tw, tid, nthr, 16);
}

// The line FFT of the per-sample passes: in FP32, radix 16 when the line has
// exactly 16 elements per thread (the launch shapes of the FP32 passes), the
// radix-4 form otherwise (FP64, and lines shorter than 16 or longer than 4096).
template <typename R, int MAXB>
__device__ __forceinline__ void line_fft(typename C2<R>::T *buf, int logN,
                                         const typename C2<R>::T *__restrict__ tw, int tid,
                                         int nthr) {
    if constexpr (sizeof(R) == 4) {
        if (nthr * 16 == (1 << logN)) {
            smem_fft16<R>(buf, logN, tw, tid, nthr);
            return;
        }
    }
    smem_fft<R, MAXB>(buf, logN, tw, tid, nthr);
}

}  // namespace sce

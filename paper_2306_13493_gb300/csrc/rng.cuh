// Normal generator of Algorithm 1 step 4(a): Philox4x32-10 + Box-Muller.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw (SC'11): per round
// the 64-bit products M0*c0 and M1*c2 (M0 = 0xD2511F53, M1 = 0xCD9E8D57) give
// c' = (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the
// key is advanced by the Weyl increments (0x9E3779B9, 0xBB67AE85) between
// rounds.  Key (seed lo, seed hi); counter (q, sample lo, sample hi, level) for
// normals 4q .. 4q+3 of a sample.
//
// Box & Muller (1958): (u0, u1) -> r cos(2 pi u1), r sin(2 pi u1), r = sqrt(-2 ln u0).
// ln and sin/cos(pi t) are evaluated from IEEE +, -, *, / and sqrt only, with
// explicit round-to-nearest intrinsics (no contraction into FMA), so the bits
// equal those of any other IEEE implementation of the same steps:
//   ln x : x = m 2^e, m in [sqrt(1/2), sqrt(2)), f = (m-1)/(m+1), s = f^2,
//          ln x = e ln2 + 2 f sum_k s^k/(2k+1)   (k <= 10 FP64, k <= 4 FP32)
//   sincos(pi t): q = rint(2t), r = t - q/2 (exact), x = pi r, Taylor series
//          of sin to x^19 / cos to x^18 (FP64, nested), x^9 / x^10 (FP32,
//          Horner form with the coefficients rounded to float32 once).
#pragma once

#include <stdint.h>

namespace sce {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t level, uint64_t sample,
                                              uint32_t q) {
    return philox4x32_10(make_uint4(q, (uint32_t)sample, (uint32_t)(sample >> 32), level),
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

// ------------------------------------------------------------------ FP64
__device__ __forceinline__ double ln_f64(double x) {
    int ei;
    double m = frexp(x, &ei);
    double e = (double)ei;
    if (m < 0.7071067811865476) {
        m = __dmul_rn(m, 2.0);
        e = __dsub_rn(e, 1.0);
    }
    const double f = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double s = __dmul_rn(f, f);
    double p = 1.0 / 21.0;
    p = __dadd_rn(1.0 / 19.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 17.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 15.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 13.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 11.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 9.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 7.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 5.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0 / 3.0, __dmul_rn(s, p));
    p = __dadd_rn(1.0, __dmul_rn(s, p));
    const double t = __dmul_rn(f, p);
    return __dadd_rn(__dmul_rn(e, 0.6931471805599453), __dadd_rn(t, t));
}

__device__ __forceinline__ void sincospi_f64(double t, double *sn, double *cs) {
    const double q = rint(__dmul_rn(t, 2.0));
    const double r = __dsub_rn(t, __dmul_rn(q, 0.5));
    const int qi = ((int)q) & 3;
    const double x = __dmul_rn(3.141592653589793, r);
    const double x2 = __dmul_rn(x, x);
    // sin: 1 - x^2/(2k(2k+1)) (...), k = 9..1
    double S = 1.0;
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 342.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 272.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 210.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 156.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 110.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 72.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 42.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 20.0));
    S = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, S), 1.0 / 6.0));
    // cos: 1 - x^2/((2k-1)2k) (...), k = 9..1
    double C = 1.0;
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 306.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 240.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 182.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 132.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 90.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 56.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 30.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 12.0));
    C = __dsub_rn(1.0, __dmul_rn(__dmul_rn(x2, C), 1.0 / 2.0));
    S = __dmul_rn(x, S);
    switch (qi) {
        case 0: *sn = S; *cs = C; break;
        case 1: *sn = C; *cs = -S; break;
        case 2: *sn = -S; *cs = -C; break;
        default: *sn = -C; *cs = S; break;
    }
}

// Normals 4q .. 4q+3 of one sample (FP64 spec).
__device__ __forceinline__ void normals4_f64(uint4 w, double out[4]) {
    const double u0 = __dmul_rn(__dadd_rn((double)w.x, 0.5), 0x1p-32);
    const double u1 = __dmul_rn(__dadd_rn((double)w.y, 0.5), 0x1p-32);
    const double u2 = __dmul_rn(__dadd_rn((double)w.z, 0.5), 0x1p-32);
    const double u3 = __dmul_rn(__dadd_rn((double)w.w, 0.5), 0x1p-32);
    double s, c;
    double r = __dsqrt_rn(__dmul_rn(-2.0, ln_f64(u0)));
    sincospi_f64(__dmul_rn(2.0, u1), &s, &c);
    out[0] = __dmul_rn(r, c);
    out[1] = __dmul_rn(r, s);
    r = __dsqrt_rn(__dmul_rn(-2.0, ln_f64(u2)));
    sincospi_f64(__dmul_rn(2.0, u3), &s, &c);
    out[2] = __dmul_rn(r, c);
    out[3] = __dmul_rn(r, s);
}

// ------------------------------------------------------------------ FP32
__device__ __forceinline__ float ln_f32(float x) {
    int ei;
    float m = frexpf(x, &ei);
    float e = (float)ei;
    if (m < 0.70710677f) {
        m = __fmul_rn(m, 2.0f);
        e = __fsub_rn(e, 1.0f);
    }
    const float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s = __fmul_rn(f, f);
    // atanh(f)/f = 1 + s/3 + s^2/5 + s^3/7 + s^4/9 (the s^5/11 term is below
    // 2^-30 of the result for |f| <= 0.1716), float32 coefficients
    float p = 0x1.c71c72p-4f;                          // 1/9
    p = __fadd_rn(0x1.24924ap-3f, __fmul_rn(s, p));    // 1/7
    p = __fadd_rn(0x1.99999ap-3f, __fmul_rn(s, p));    // 1/5
    p = __fadd_rn(0x1.555556p-2f, __fmul_rn(s, p));    // 1/3
    p = __fadd_rn(1.0f, __fmul_rn(s, p));
    const float t = __fmul_rn(f, p);
    return __fadd_rn(__fmul_rn(e, 0.6931472f), __fadd_rn(t, t));
}

__device__ __forceinline__ void sincospi_f32(float t, float *sn, float *cs) {
    const float q = rintf(__fmul_rn(t, 2.0f));
    const float r = __fsub_rn(t, __fmul_rn(q, 0.5f));
    const int qi = ((int)q) & 3;
    const float x = __fmul_rn(3.1415927f, r);
    const float x2 = __fmul_rn(x, x);
    // Taylor polynomials for |x| <= pi/4 in Horner form with float32
    // coefficients (-1)^k/(2k+1)! and (-1)^k/(2k)!: sin to x^9, cos to x^10
    // (the next terms are below 2e-9)
    float S = 0x1.71de3ap-19f;                          // 1/9!
    S = __fadd_rn(-0x1.a01a02p-13f, __fmul_rn(x2, S));  // -1/7!
    S = __fadd_rn(0x1.111112p-7f, __fmul_rn(x2, S));    // 1/5!
    S = __fadd_rn(-0x1.555556p-3f, __fmul_rn(x2, S));   // -1/3!
    S = __fadd_rn(1.0f, __fmul_rn(x2, S));
    float C = -0x1.27e4fcp-22f;                         // -1/10!
    C = __fadd_rn(0x1.a01a02p-16f, __fmul_rn(x2, C));   // 1/8!
    C = __fadd_rn(-0x1.6c16c2p-10f, __fmul_rn(x2, C));  // -1/6!
    C = __fadd_rn(0x1.555556p-5f, __fmul_rn(x2, C));    // 1/4!
    C = __fadd_rn(-0.5f, __fmul_rn(x2, C));             // -1/2!
    C = __fadd_rn(1.0f, __fmul_rn(x2, C));
    S = __fmul_rn(x, S);
    switch (qi) {
        case 0: *sn = S; *cs = C; break;
        case 1: *sn = C; *cs = -S; break;
        case 2: *sn = -S; *cs = -C; break;
        default: *sn = -C; *cs = S; break;
    }
}

__device__ __forceinline__ void normals4_f32(uint4 w, float out[4]) {
    const float u0 = __fmul_rn(__fadd_rn(__uint2float_rn(w.x), 0.5f), 0x1p-32f);
    const float u1 = __fmul_rn(__fadd_rn(__uint2float_rn(w.y), 0.5f), 0x1p-32f);
    const float u2 = __fmul_rn(__fadd_rn(__uint2float_rn(w.z), 0.5f), 0x1p-32f);
    const float u3 = __fmul_rn(__fadd_rn(__uint2float_rn(w.w), 0.5f), 0x1p-32f);
    float s, c;
    float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_f32(u0)));
    sincospi_f32(__fmul_rn(2.0f, u1), &s, &c);
    out[0] = __fmul_rn(r, c);
    out[1] = __fmul_rn(r, s);
    r = __fsqrt_rn(__fmul_rn(-2.0f, ln_f32(u2)));
    sincospi_f32(__fmul_rn(2.0f, u3), &s, &c);
    out[2] = __fmul_rn(r, c);
    out[3] = __fmul_rn(r, s);
}

template <typename R> struct Normals;
template <> struct Normals<double> {
    static __device__ __forceinline__ void gen4(uint4 w, double o[4]) { normals4_f64(w, o); }
};
template <> struct Normals<float> {
    static __device__ __forceinline__ void gen4(uint4 w, float o[4]) { normals4_f32(w, o); }
};

}  // namespace sce

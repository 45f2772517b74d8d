// Float-float ("double-single") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, carrying ~48 bits.
// Built from the error-free transformations of Knuth (TwoSum, TAOCP vol. 2,
// §4.2.2) and Dekker (FastTwoSum; TwoProduct, here with a fused multiply-add
// giving the exact rounding error of a product), as in the double-double
// algorithms of Hida, Li and Bailey (2001) with FP32 in place of FP64.
//
// On GB300 FP64 runs at ~1/64 of the FP32 rate, so the refinement residual of
// the mixed-precision solver uses these FP32 operations instead of FP64 ones.
// The transformations use explicit round-to-nearest intrinsics so that no
// operation is contracted or reassociated.
#pragma once

namespace sce {

struct ff {
    float hi, lo;
};

// s + e = a + b exactly (any a, b)
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly, given |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_from(float a) { return {a, 0.0f}; }

// hi + lo of a double, rounded to the nearest float-float
__device__ __forceinline__ ff ff_from_double(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

}  // namespace sce

// df32.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers (about 48 significant bits).  Built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2) and TwoProduct via a fused
// multiply-add (Dekker 1971; an FMA gives the product's rounding error
// exactly), combined as in the double-double algorithms of Hida, Li and
// Bailey (2001).  Every operation uses the explicitly rounded intrinsics so
// the compiler cannot contract or reorder the error terms.
//
// Used where FP64 accuracy is needed at FP32-pipe cost: the HMC action S(psi)
// and kinetic energy on GB300, whose FP64 rate is a small fraction of FP32.
#pragma once
#include <cuda_runtime.h>

namespace ihmc {

struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return f2{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return f2{s, e};
}

__device__ __forceinline__ f2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return f2{p, e};
}

__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
    const f2 s = two_sum(a.hi, b.hi);
    const f2 t = two_sum(a.lo, b.lo);
    const f2 u = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ f2 df_add_f(f2 a, float b) {
    const f2 s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ f2 df_neg(f2 a) { return f2{-a.hi, -a.lo}; }

__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ f2 df_mul_f(f2 a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ f2 df_from_double(double x) {
    const float hi = (float)x;
    return f2{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ double df_to_double(f2 a) { return (double)a.hi + (double)a.lo; }

// Table of g(y) = log(1 + exp(-y)) on y_k = k/16, k = 0 .. LOG1PEXP_K, as
// Taylor coefficients c_n = g^(n)(y_k)/n!, n = 0..7: c0, c1, c2 as double-
// floats and c3..c7 as floats, packed into three float4 per node:
//   {c0.hi, c0.lo, c1.hi, c1.lo}, {c2.hi, c2.lo, c3, c4}, {c5, c6, c7, 0}.
// For y >= 36, g(y) < 2.4e-16 and is taken as exp(-y).
constexpr int LOG1PEXP_PER_UNIT = 16;
constexpr int LOG1PEXP_K = 36 * LOG1PEXP_PER_UNIT;

// g(y) for y >= 0 given as a double-float; absolute error below 1e-13 (the
// FP32 rounding of c3 times d^3 dominates).
__device__ __forceinline__ f2 log1pexp_neg(f2 y, const float4 *__restrict__ tab) {
    if (y.hi >= 36.0f) return f2{__expf(-y.hi), 0.0f};
    const int k = __float2int_rn(y.hi * (float)LOG1PEXP_PER_UNIT);
    // y.hi - k/16 is exact (Sterbenz), the low word carries the rest
    const f2 d = fast_two_sum(__fsub_rn(y.hi, (float)k * (1.0f / LOG1PEXP_PER_UNIT)), y.lo);
    const float4 q0 = __ldg(tab + 3 * k);
    const float4 q1 = __ldg(tab + 3 * k + 1);
    const float4 q2 = __ldg(tab + 3 * k + 2);
    const float dh = d.hi;
    float r = fmaf(dh, q2.z, q2.y);   // c6 + d c7
    r = fmaf(dh, r, q2.x);            // c5 + d (...)
    r = fmaf(dh, r, q1.w);            // c4 + ...
    r = fmaf(dh, r, q1.z);            // c3 + ...
    f2 t = df_add_f(f2{q1.x, q1.y}, __fmul_rn(dh, r));  // c2 + d r
    t = df_add(f2{q0.z, q0.w}, df_mul(d, t));            // c1 + d t
    return df_add(f2{q0.x, q0.y}, df_mul(d, t));          // c0 + d t
}

}  // namespace ihmc

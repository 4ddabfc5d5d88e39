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

// Quicker sum (one TwoSum, the low words added in FP32): its error is a few
// units of 2^-48 of max(|a|, |b|) in absolute terms -- the accuracy the action
// sums need -- though not relative to a small result.
__device__ __forceinline__ f2 df_add_q(f2 a, f2 b) {
    const f2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
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

// Accumulators: a double-float high part plus an FP32 sum of the addends' low
// words (their magnitude is ~2^-24 of the terms).
__device__ __forceinline__ void acc_add(f2 &hi, float &lo, f2 v) {
    hi = df_add_f(hi, v.hi);
    lo = __fadd_rn(lo, v.lo);
}
__device__ __forceinline__ double acc_val(f2 hi, float lo) { return df_to_double(hi) + (double)lo; }

// Kahan (1965) compensated summation in FP32.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}
__device__ __forceinline__ double kahan_val(float s, float c) { return (double)s - (double)c; }

// Table of g(y) = log(1 + exp(-y)) on y_k = k/32, k = 0 .. LOG1PEXP_K: one
// float4 per node {g(y_k).hi, g(y_k).lo, s.hi, s.lo} with s = 1/(1 + e^{y_k}).
// With w = s(1-s) and v = 1-2s the derivatives are polynomials in s
// (g' = -s, ds/dy = -w):
//   g1 = -s, g2 = w, g3 = -w v, g4 = w(1-6w), g5 = -w v(1-12w),
//   g6 = w(1-30w+120w^2),
// and g(y_k + d) = sum_n g_n d^n / n!, |d| <= 1/64; the next term is below
// 2e-17.  g0 and the first-order term are kept as double-floats; the second to
// sixth orders (together below 3.1e-5) in FP32.  For y >= 36, g(y) < 2.4e-16
// and is taken as exp(-y).
constexpr int LOG1PEXP_PER_UNIT = 32;
constexpr int LOG1PEXP_K = 36 * LOG1PEXP_PER_UNIT;

// g(y) for y >= 0 given as a double-float; absolute error below 1e-11.
// tab may live in shared or global memory.
__device__ __forceinline__ f2 log1pexp_neg(f2 y, const float4 *tab) {
    if (y.hi >= 36.0f) return f2{__expf(-y.hi), 0.0f};
    const int k = __float2int_rn(y.hi * (float)LOG1PEXP_PER_UNIT);
    // y.hi - k/32 is exact (Sterbenz), the low word carries the rest
    const f2 d = two_sum(__fsub_rn(y.hi, (float)k * (1.0f / LOG1PEXP_PER_UNIT)), y.lo);
    const float4 q = tab[k];
    const f2 g0{q.x, q.y}, s{q.z, q.w};
    const f2 t1 = df_mul(df_neg(s), d);   // g1 d, double-float
    // second to sixth order in FP32 (Horner in d)
    const float wf = fmaf(-s.hi, s.hi, s.hi), vf = fmaf(-2.0f, s.hi, 1.0f), dh = d.hi;
    const float c2 = 0.5f * wf;
    const float c3 = -wf * vf * (1.0f / 6.0f);
    const float c4 = wf * fmaf(-6.0f, wf, 1.0f) * (1.0f / 24.0f);
    const float c5 = -wf * vf * fmaf(-12.0f, wf, 1.0f) * (1.0f / 120.0f);
    const float c6 = wf * fmaf(wf, fmaf(120.0f, wf, -30.0f), 1.0f) * (1.0f / 720.0f);
    const float r = fmaf(dh, fmaf(dh, fmaf(dh, fmaf(dh, c6, c5), c4), c3), c2);
    return df_add_q(g0, df_add_f(t1, dh * dh * r));
}

}  // namespace ihmc

// Double-float ("FP32 pair") arithmetic for the compensated residual recompute.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers.  The error-free
// transformations are the classical ones: TwoSum (Knuth, TAOCP vol. 2),
// Fast2Sum (Dekker 1971) and the FMA form of TwoProd; the double-float add and
// multiply follow Dekker's composition.  All arithmetic stays in FP32; nvcc
// does not reassociate additions, and every product whose rounding error is
// needed is taken explicitly through fmaf.
#pragma once

namespace ap {
namespace df {

struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
    F2 s = two_sum(a.h, b.h);
    const float e = s.l + (a.l + b.l);
    return fast_two_sum(s.h, e);
}

__device__ __forceinline__ F2 add_f(F2 a, float b) {
    F2 s = two_sum(a.h, b);
    return fast_two_sum(s.h, s.l + a.l);
}

__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    F2 p = two_prod(a.h, b.h);
    const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
    return fast_two_sum(p.h, e);
}

__device__ __forceinline__ F2 mul_f(F2 a, float b) {
    F2 p = two_prod(a.h, b);
    return fast_two_sum(p.h, fmaf(a.l, b, p.l));
}

// ln 2 and log2 e as FP32 pairs (hi = nearest float, lo = remainder)
constexpr float kLn2H = 0.693147182464599609375f;
constexpr float kLn2L = -1.9046542121259336e-09f;
constexpr float kLog2eH = 1.44269502162933349609375f;
constexpr float kLog2eL = 1.925963033500011e-08f;
constexpr float kThirdH = 0.3333333432674407958984375f;
constexpr float kThirdL = -9.934107758624577e-09f;
constexpr float kSixthH = 0.16666667163372039794921875f;
constexpr float kSixthL = -4.967053879312289e-09f;

// 2^(-t) for t = t.h + t.l >= 0 with about 2^-40 relative error.
// t = k + r, k = nearest integer, |r| <= 1/2;  2^-r = e^-z, z = r ln 2, |z| < 0.35;
// e^-z = 1 - z + z^2/2 - z^3/6 + z^4 q(z): the leading terms in double-float,
// the tail q (|z^4 q| < 7e-4) in FP32 Horner form (Taylor coefficients).
__device__ __forceinline__ F2 exp2_neg(F2 t) {
    const float k = rintf(t.h);
    if (k > 125.0f) return {0.0f, 0.0f};
    const F2 r = fast_two_sum(t.h - k, t.l);
    const F2 z = mul(r, F2{kLn2H, kLn2L});
    const float zh = z.h;
    float q = -1.0f / 362880.0f;
    q = fmaf(q, zh, 1.0f / 40320.0f);
    q = fmaf(q, zh, -1.0f / 5040.0f);
    q = fmaf(q, zh, 1.0f / 720.0f);
    q = fmaf(q, zh, -1.0f / 120.0f);
    q = fmaf(q, zh, 1.0f / 24.0f);
    // Horner in double-float: ((q z - 1/6) z + 1/2) z - 1) z + 1
    F2 acc = mul_f(z, q);
    acc = add(acc, F2{-kSixthH, -kSixthL});
    acc = mul(acc, z);
    acc = add_f(acc, 0.5f);
    acc = mul(acc, z);
    acc = add_f(acc, -1.0f);
    acc = mul(acc, z);
    acc = add_f(acc, 1.0f);
    // scale by 2^-k exactly (k <= 125 keeps the result normal or zero)
    const float sc = __int_as_float((127 - (int)k) << 23);
    return {acc.h * sc, acc.l * sc};
}

// sqrt of a double-float t >= 0: IEEE sqrt of t.h plus one Newton correction.
__device__ __forceinline__ F2 sqrt_df(F2 t) {
    if (t.h <= 0.0f) return {0.0f, 0.0f};
    const float s = __fsqrt_rn(t.h);
    const F2 ss = two_prod(s, s);
    const float corr = ((t.h - ss.h) - ss.l + t.l) * (0.5f / s);
    return fast_two_sum(s, corr);
}

}  // namespace df
}  // namespace ap

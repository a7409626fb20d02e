// Double-float arithmetic for the extended-precision heterodyne (mbh_hetx.cu): complex values,
// sine and cosine, exp and sin(y)/y of double-float arguments, built on the error-free
// primitives of mbh_df.cuh.  Everything runs on the float32 pipe (B300's float64 pipe is 1/64
// of its float32 rate).
//
// Results are "lazy" double-floats: hi + lo unevaluated, lo not renormalised (|lo| a few ulp of
// hi at most), relative error ~2^-45 per operation; the callers renormalise where a value is
// compared.  What the heterodyne needs is absolute accuracy on O(1) quantities (~1e-9 per edge
// at SNR 1000): the Taylor tails below keep in float32 only the terms whose float32 rounding
// stays under ~1e-10 absolute, and everything else in double-float.
#pragma once
#include <cuda_runtime.h>

#include "mbh_df.cuh"

namespace mbh {

struct c2f {
    f2 re, im;
};

__device__ __forceinline__ f2 dd_scale(f2 a, float s) { return {a.hi * s, a.lo * s}; }   // s a power of two
__device__ __forceinline__ f2 dd_sub_lazy(f2 a, f2 b) { return dd_add_lazy(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ f2 dd_add_f_lazy(f2 a, float b)
{
    const f2 s = two_sum(a.hi, b);
    return {s.hi, __fadd_rn(s.lo, a.lo)};
}
__device__ __forceinline__ f2 dd_mul_f_lazy(f2 a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    return {p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p))};
}
__device__ __forceinline__ f2 dd_sqr_lazy(f2 a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    return {p, __fmaf_rn(2.0f * a.hi, a.lo, __fmaf_rn(a.hi, a.hi, -p))};
}
__device__ __forceinline__ f2 dd_norm(f2 a) { return fast_two_sum(a.hi, a.lo); }
// a b + c and a b keeping the a.lo b.lo term: along a chain of products of correlated
// operands (a Horner evaluation of c_0 v^-5) the dropped terms share a sign and add up to a
// bias of ~(lo/hi)^2 per step, ~1e-9 rad at |Psi| ~ 1e6
__device__ __forceinline__ f2 dd_fma_full(f2 a, f2 b, f2 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.lo, b.lo, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
    const f2 s = two_sum(p, c.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo))};
}
__device__ __forceinline__ f2 dd_mul_full(f2 a, f2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    return {p, __fmaf_rn(a.lo, b.lo, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p))))};
}

// a^2 with the lo^2 term (for operands that may be unnormalised)
__device__ __forceinline__ f2 dd_sqr_full(f2 a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    return {p, __fmaf_rn(a.lo, a.lo, __fmaf_rn(2.0f * a.hi, a.lo, __fmaf_rn(a.hi, a.hi, -p)))};
}
__device__ __forceinline__ f2 dd_from(float a) { return {a, 0.0f}; }

__device__ __forceinline__ c2f cd_add(c2f a, c2f b) { return {dd_add_lazy(a.re, b.re), dd_add_lazy(a.im, b.im)}; }
__device__ __forceinline__ c2f cd_sub(c2f a, c2f b) { return {dd_sub_lazy(a.re, b.re), dd_sub_lazy(a.im, b.im)}; }
__device__ __forceinline__ c2f cd_scale(c2f a, float s) { return {dd_scale(a.re, s), dd_scale(a.im, s)}; }
__device__ __forceinline__ c2f cd_mul_r(c2f a, f2 b) { return {dd_mul_lazy(a.re, b), dd_mul_lazy(a.im, b)}; }
__device__ __forceinline__ c2f cd_mul_f(c2f a, float b) { return {dd_mul_f_lazy(a.re, b), dd_mul_f_lazy(a.im, b)}; }
__device__ __forceinline__ c2f cd_mul(c2f a, c2f b)
{
    return {dd_sub_lazy(dd_mul_lazy(a.re, b.re), dd_mul_lazy(a.im, b.im)),
            dd_add_lazy(dd_mul_lazy(a.re, b.im), dd_mul_lazy(a.im, b.re))};
}
__device__ __forceinline__ c2f cd_norm(c2f a) { return {dd_norm(a.re), dd_norm(a.im)}; }

// ---- sine and cosine ---------------------------------------------------------------------
// 2 pi and pi/16 as three floats (Cody-Waite): the first term's products with the integers used
// below are exact inside an FMA (see dd_reduce_2pi and dd_sincos), the second enters through an
// exact two-product.
constexpr double kTwoPiD = 6.283185307179586476925286766559005768;
// 2 pi = P2a + P2b + P2c to ~4e-23, the three parts rounded from a 60-digit value of 2 pi (the
// float64 value of 2 pi is itself 2.4e-16 off, which over the ~1e6 turns of a 1e7-rad phase would
// be a systematic 5e-10 rad)
constexpr float kP2a = 0x1.921fb6p+2f;
constexpr float kP2b = -0x1.777a5cp-23f;
constexpr float kP2c = -0x1.ee59dap-48f;
constexpr double kPi16D = 0.196349540849362077403915211455980405;
constexpr float kQ16a = (float)kPi16D;
constexpr float kQ16b = (float)(kPi16D - (double)kQ16a);
constexpr float kQ16c = (float)(kPi16D - (double)kQ16a - (double)kQ16b);

// x - n 2 pi with n = round(x / 2 pi) (|n| < 2^22).  The first step x_hi - n P2a is exact: its
// exact value is a multiple of ulp(P2a) = 2^-21 (and of ulp(x_hi) >= 2^-21 whenever n != 0)
// below 8 in magnitude.  n comes from a float32 product, whose rounding (~6e-8 |x|/2 pi) can
// miss the nearest integer by one once |x| exceeds ~1e5; a second step with n2 in {-1, 0, 1}
// (exact, and the identity when n2 = 0) brings the result within pi (1 + 2^-20).
__device__ __forceinline__ f2 dd_reduce_2pi_step(f2 x)
{
    const float n = rintf(x.hi * (float)(1.0 / kTwoPiD));
    const float r = __fmaf_rn(-n, kP2a, x.hi);
    const float p = __fmul_rn(n, kP2b);
    const float e = __fmaf_rn(n, kP2b, -p);
    const f2 s = two_sum(r, -p);
    // renormalised: x.lo (up to ulp(x.hi)/2, ~0.06 at |x| ~ 2e6) can exceed the reduced value's
    // own ulp, and the small-angle forms below read only the high word
    return two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, x.lo), __fmaf_rn(-n, kP2c, -e)));
}

__device__ __forceinline__ f2 dd_reduce_2pi(f2 x) { return dd_reduce_2pi_step(dd_reduce_2pi_step(x)); }

// a b - n 2 pi for a double-float a and a triple-float b = b.hi + b.lo + bx, |a b| < 2^22 pi
// (n = round(a.hi b.hi / 2 pi); the result lies within ~pi + 1.5 of zero, as a normalised
// double-float good to ~1e-14).  At |a b| ~ 1e6-1e7 the low word of a plain double-float
// product resolves ~|a b| 2^-48 ~ 1e-8: the product's small terms (a.lo b.lo, a.hi bx, the
// residuals of the partial products) fall below it and round away, alike at every a for a
// constant b.  Here the leading product is taken exactly, reduced first (exactly, as in
// dd_reduce_2pi_step), and the O(1) partial products and the small terms are added after.
__device__ __forceinline__ f2 dd_mul_mod2pi(f2 a, f2 b, float bx)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);           // p + e = a.hi b.hi
    const float n = rintf(p * (float)(1.0 / kTwoPiD));
    const float r = __fmaf_rn(-n, kP2a, p);              // exact
    const float q = __fmul_rn(n, kP2b);
    const float qe = __fmaf_rn(n, kP2b, -q);             // q + qe = n P2b
    const float t1 = __fmul_rn(a.hi, b.lo);
    const float t1e = __fmaf_rn(a.hi, b.lo, -t1);        // t1 + t1e = a.hi b.lo
    const float t2 = __fmul_rn(a.lo, b.hi);
    const float t2e = __fmaf_rn(a.lo, b.hi, -t2);        // t2 + t2e = a.lo b.hi
    const f2 s0 = two_sum(r, -q);
    const f2 s1 = two_sum(s0.hi, e);
    const f2 s2 = two_sum(s1.hi, t1);
    const f2 s3 = two_sum(s2.hi, t2);
    // the words below: the two-sums' residuals (each below ulp(~pi)/2) and the small terms
    float lo = __fadd_rn(__fadd_rn(s0.lo, s1.lo), __fadd_rn(s2.lo, s3.lo));
    float sm = __fmaf_rn(a.lo, b.lo, __fmaf_rn(a.hi, bx, __fadd_rn(t1e, t2e)));
    sm = __fsub_rn(sm, __fmaf_rn(n, kP2c, qe));
    return two_sum(s3.hi, __fadd_rn(lo, sm));
}

// sin a and cos a - 1 for |a| <= 0.1 (a double-float): sin a = a + a^3 (-1/6 + a^2/120 -
// a^4/5040 + a^6/362880) with the a^3 term in float32 (its four float32 roundings, ~2e-7 of
// |a|^3/6, are below 3.5e-11 at 0.1; at 0.19 they reached 1.7e-10),
// cos a - 1 = -a^2/2 (double-float) + a^4 (1/24 - a^2/720 + a^4/40320) (float32 tail < 4e-5).
__device__ __forceinline__ void dd_sincos_small(f2 a, f2& s, f2& cm1)
{
    const float a2 = a.hi * a.hi;
    const float st = a.hi * a2 * fmaf(a2, fmaf(a2, fmaf(a2, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f),
                                      -1.0f / 6.0f);
    s = dd_add_f_lazy(a, st);
    const f2 sq = dd_sqr_lazy(a);
    const float ct = a2 * a2 * fmaf(a2, fmaf(a2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f);
    cm1 = {-0.5f * sq.hi, fmaf(-0.5f, sq.lo, ct)};
}

// Table of sin(k pi/16) and cos(k pi/16) - 1, k = 0..16, as double-floats: (s hi, s lo, c hi,
// c lo).  Filled from float64 literals (40-digit values rounded to float64, then split).
struct SinTab {
    float4 v[17];
};

// sin r and cos r - 1 for |r| <= pi (1 + 2^-20): k = round(|r| 16/pi), a = |r| - k pi/16
// (|a| <= pi/32; the first step exact, as in dd_reduce_2pi), the small-angle forms of a, then
// sin r = S_k + sin a + S_k (cos a - 1) + (C_k - 1) sin a and
// cos r - 1 = (C_k - 1) + (cos a - 1) + (C_k - 1)(cos a - 1) - S_k sin a, sign of r restored.
__device__ __forceinline__ void dd_sincos(f2 r, const SinTab& tab, f2& s, f2& cm1)
{
    const bool neg = r.hi < 0.0f;
    const f2 ar = neg ? f2{-r.hi, -r.lo} : r;
    // k <= 16 for |r| <= pi (1 + 2^-20); the bound also keeps the table read in range for any
    // input (a non-finite or unreduced argument gives a wrong value, never a stray read)
    const float k = fminf(rintf(ar.hi * (float)(16.0 / 3.141592653589793238462643383279502884)), 16.0f);
    const float a0 = __fmaf_rn(-k, kQ16a, ar.hi);
    const float p = __fmul_rn(k, kQ16b);
    const float e = __fmaf_rn(k, kQ16b, -p);
    const f2 t = two_sum(a0, -p);
    const f2 a = two_sum(t.hi, __fadd_rn(__fadd_rn(t.lo, ar.lo), __fmaf_rn(-k, kQ16c, -e)));
    f2 sa, ca;
    dd_sincos_small(a, sa, ca);
    const float4 T = tab.v[(int)k];
    const f2 Sk = {T.x, T.y}, Ck = {T.z, T.w};
    s = dd_add_lazy(dd_add_lazy(Sk, sa), dd_add_lazy(dd_mul_lazy(Sk, ca), dd_mul_lazy(Ck, sa)));
    cm1 = dd_add_lazy(dd_add_lazy(Ck, ca), dd_sub_lazy(dd_mul_lazy(Ck, ca), dd_mul_lazy(Sk, sa)));
    if (neg) s = {-s.hi, -s.lo};
}

// sin x and cos x - 1 of any double-float |x| < 2^22 pi (reduction by 2 pi, then dd_sincos).
// x is renormalised first: arguments from lazy arithmetic after a cancellation (an orbit angle
// (t - t_ref) 2 pi/yr with t ~ t_ref ~ 3e7 s) can carry a low word of many ulps of the high
// word, which the small-angle series would miss in its cubic term (~a^2/2 lo, 4e-9 at 0.2).
__device__ __forceinline__ void dd_sincos_any(f2 x, const SinTab& tab, f2& s, f2& cm1)
{
    x = two_sum(x.hi, x.lo);
    if (fabsf(x.hi) <= 0.1f) {
        dd_sincos_small(x, s, cm1);
        return;
    }
    dd_sincos(fabsf(x.hi) > 3.14f ? dd_reduce_2pi(x) : x, tab, s, cm1);
}

// ---- exp -----------------------------------------------------------------------------------
constexpr double kLn2D = 0.693147180559945309417232121458176568;
constexpr float kL2a = (float)kLn2D;
constexpr float kL2b = (float)(kLn2D - (double)kL2a);
constexpr float kL2c = (float)(kLn2D - (double)kL2a - (double)kL2b);
constexpr f2 kInv6 = df_const(1.0 / 6.0);

// exp(u) for |u| <= 60: n = round(u/ln 2), a = u - n ln 2 (|a| <= 0.35; first step exact as
// above), exp(a) = 1 + a + a^2/2 + a^3/6 + a^4 p(a) with the quartic tail in float32 (its
// rounding < 4e-11), times 2^n (exact).
__device__ __forceinline__ f2 dd_exp(f2 u)
{
    const float n = rintf(u.hi * (float)(1.0 / kLn2D));
    const float a0 = __fmaf_rn(-n, kL2a, u.hi);
    const float p = __fmul_rn(n, kL2b);
    const float e = __fmaf_rn(n, kL2b, -p);
    const f2 t = two_sum(a0, -p);
    const f2 a = two_sum(t.hi, __fadd_rn(__fadd_rn(t.lo, u.lo), __fmaf_rn(-n, kL2c, -e)));
    const float ah = a.hi;
    float tail = fmaf(ah, 1.0f / 479001600.0f, 1.0f / 39916800.0f);
    tail = fmaf(tail, ah, 1.0f / 3628800.0f);
    tail = fmaf(tail, ah, 1.0f / 362880.0f);
    tail = fmaf(tail, ah, 1.0f / 40320.0f);
    tail = fmaf(tail, ah, 1.0f / 5040.0f);
    tail = fmaf(tail, ah, 1.0f / 720.0f);
    tail = fmaf(tail, ah, 1.0f / 120.0f);
    tail = fmaf(tail, ah, 1.0f / 24.0f);
    const float a2f = ah * ah;
    tail *= a2f * a2f;
    const f2 a2 = dd_sqr_lazy(a);
    const f2 a3_6 = dd_mul_lazy(dd_mul_lazy(a2, a), kInv6);
    f2 em1 = dd_add_lazy(a, dd_add_lazy(dd_scale(a2, 0.5f), dd_add_f_lazy(a3_6, tail)));
    f2 r = dd_add_f_lazy(em1, 1.0f);
    const float sc = __int_as_float((127 + (int)n) << 23);   // 2^n, |n| <= 87
    return {r.hi * sc, r.lo * sc};
}

// ---- sin(y)/y ------------------------------------------------------------------------------
// (-1)^j/(2j+1)!, j = 0..11
__device__ __forceinline__ float sinc_coef(int j)
{
    constexpr float c[12] = {1.0f, -1.0f / 6.0f, 1.0f / 120.0f, -1.0f / 5040.0f, 1.0f / 362880.0f,
                             -1.0f / 39916800.0f, 1.0f / 6227020800.0f, -1.0f / 1307674368000.0f,
                             1.0f / 355687428096000.0f, -1.0f / 121645100408832000.0f,
                             1.0f / 51090942171709440000.0f, -1.0f / 25852016738884976640000.0f};
    return c[j];
}

// The double-float constants (-1)^j/(2j+1)! for j = 1..4
constexpr f2 kSc1 = df_const(-1.0 / 6.0);
constexpr f2 kSc2 = df_const(1.0 / 120.0);
constexpr f2 kSc3 = df_const(-1.0 / 5040.0);
constexpr f2 kSc4 = df_const(1.0 / 362880.0);

// sin(y)/y for |y| < 2.8 as its Taylor series in y^2 to y^22/23!: terms j >= 5 (below 7e-4) in
// float32, j <= 4 by a double-float Horner step each.
__device__ __forceinline__ f2 dd_sinc_series(f2 y)
{
    const f2 y2 = dd_sqr_lazy(y);
    const float z = y2.hi;
    float t = sinc_coef(11);
#pragma unroll
    for (int j = 10; j >= 5; --j) t = fmaf(t, z, sinc_coef(j));
    f2 acc = dd_add_f_lazy(kSc4, t * z);
    acc = dd_fma_lazy(acc, y2, kSc3);
    acc = dd_fma_lazy(acc, y2, kSc2);
    acc = dd_fma_lazy(acc, y2, kSc1);
    return dd_add_f_lazy(dd_mul_lazy(acc, y2), 1.0f);
}

// q = a / b for double-floats (b != 0): one float32 quotient and one correction step.
__device__ __forceinline__ f2 dd_div(f2 a, f2 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const f2 r = dd_sub_lazy(a, dd_mul_f_lazy(b, q1));
    const float q2 = __fdiv_rn(__fadd_rn(r.hi, r.lo), b.hi);
    return fast_two_sum(q1, q2);
}

// sin(y)/y for any double-float y
__device__ __forceinline__ f2 dd_sinc(f2 y, const SinTab& tab)
{
    if (fabsf(y.hi) < 2.8f) return dd_sinc_series(y);
    f2 s, c;
    dd_sincos_any(y, tab, s, c);
    return dd_div(s, y);
}

}  // namespace mbh

// Double-float ("df") arithmetic: float64-class results on B300's float32 and integer pipes.
//
// B300 executes float64 FMA at 2 per SM per clock, 1/64 of float32 (measured 566 G/s against
// 34.6 T/s), and its float64 pipe also carries conversions, compares and rounding.  A value is
// kept as an unevaluated sum hi + lo of two floats (~48 significant bits); products use the
// FMA two-product, sums Knuth's two-sum.  All primitives use the _rn intrinsics so that the
// compiler cannot contract a product into a following add, which would break the error-free
// transformations.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mbh {

struct f2 {
    float hi, lo;
};

// exact split of a double constant (host or device, compile time)
__host__ __device__ constexpr f2 df_const(double x)
{
    return {(float)x, (float)(x - (double)(float)x)};
}

// x * 2^-sh as hi + lo (relative error <= 2^-47) with integer operations only.  Zero,
// denormals and magnitudes below 2^-75 (after scaling) map to 0; the caller picks sh so that
// |x| 2^-sh stays below 2^127.
__device__ __forceinline__ f2 split_f64(double x, int sh)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((u >> 52) & 0x7ffu);
    const int fe = e - 1023 + 127 - sh;
    if (e == 0 || fe <= 52) return {0.0f, 0.0f};
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
    const unsigned hib = sign | ((unsigned)fe << 23) | (unsigned)(mant >> 29);
    const unsigned rem = (unsigned)(mant & 0x1FFFFFFFull);
    const float lo = __fmul_rn(__uint2float_rn(rem), __int_as_float((fe - 52) << 23));  // rem 2^(fe-179)
    return {__int_as_float((int)hib), __int_as_float(__float_as_int(lo) | (int)sign)};
}

// s + e = a + b exactly
__device__ __forceinline__ f2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ f2 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ f2 dd_add(f2 a, f2 b)
{
    f2 s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ f2 dd_neg(f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ f2 dd_sub(f2 a, f2 b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ f2 dd_add_f(f2 a, float b)
{
    f2 s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ f2 dd_mul(f2 a, f2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ f2 dd_mul_f(f2 a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}

// a * b + c; the product is left unnormalised (p + e with |e| <= ulp(p)), which the
// two-sum at the start of dd_add absorbs.
__device__ __forceinline__ f2 dd_fma(f2 a, f2 b, f2 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return dd_add({p, e}, c);
}

// a * b + c without the final renormalisation: hi is the rounded sum of the product's and c's
// high parts, lo collects the exact two-sum error and the low-order terms (|lo| may exceed
// ulp(hi)/2 by a little).  Chained Horner steps accept such operands unchanged (every product
// and sum of high parts is still exact), and so does dd_mul, which normalises its result.
__device__ __forceinline__ f2 dd_fma_lazy(f2 a, f2 b, f2 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    const f2 s = two_sum(p, c.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo))};
}

// a * b and a + b without the final renormalisation, for operands of further dd_* arithmetic
// (not for the comparisons dd_le / dd_lt0, which need normalised values)
__device__ __forceinline__ f2 dd_mul_lazy(f2 a, f2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return {p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e))};
}

__device__ __forceinline__ f2 dd_add_lazy(f2 a, f2 b)
{
    const f2 s = two_sum(a.hi, b.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ float dd_to_float(f2 a) { return __fadd_rn(a.hi, a.lo); }

// a <= b for df values normalised with round-to-nearest (|lo| <= ulp(hi)/2): the order of
// the (hi, lo) pairs is the order of the values
__device__ __forceinline__ bool dd_le(f2 a, f2 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// sign test of a (normalised) df value
__device__ __forceinline__ bool dd_le0(f2 a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo <= 0.0f); }
__device__ __forceinline__ bool dd_lt0(f2 a) { return a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f); }

// ---- unnormalised accumulation used by the streaming reduction --------------------------
// a * b with a, b as (hi, lo): hi*hi exactly as p + e, plus the cross terms (not normalised).
__device__ __forceinline__ f2 df_mul(f2 a, f2 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);
    return {p, __fadd_rn(e, __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi)))};
}

__device__ __forceinline__ f2 df_sqr(f2 a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    const float e = __fmaf_rn(a.hi, a.hi, -p);
    return {p, __fmaf_rn(2.0f * a.hi, a.lo, e)};
}

// s += x with the two-sum on the high parts; low parts and the rounding error go to s.lo.
__device__ __forceinline__ void df_acc(f2& s, f2 x)
{
    const f2 t = two_sum(s.hi, x.hi);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, x.lo));
}

__device__ __forceinline__ f2 df_add(f2 a, f2 b)
{
    f2 s = a;
    df_acc(s, b);
    return s;
}

__device__ __forceinline__ double df_to_double(f2 a) { return (double)a.hi + (double)a.lo; }

}  // namespace mbh

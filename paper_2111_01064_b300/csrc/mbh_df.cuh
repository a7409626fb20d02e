// Double-float ("df") helpers: float64-class arithmetic on B300's float32 and integer pipes.
//
// B300 executes float64 FMA at 2 per SM per clock (1/64 of float32), so even a streaming
// reduction that does five float64 operations per complex element is bound by the float64
// pipe at ~1.8 TB/s, far below HBM.  Here a float64 input x is split exactly, with integer
// operations only, into floats hi + lo = x * 2^-sh (hi: sign, exponent and the top 23
// mantissa bits; lo: the remaining 29 bits, rounded to 24); products use the FMA two-product
// and sums the two-sum, so results carry ~47 bits without touching the float64 unit.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mbh {

struct f2 {
    float hi, lo;
};

// x * 2^-sh as hi + lo (relative error <= 2^-47).  Zero, denormals and magnitudes below
// 2^-75 (after scaling) map to 0; the caller picks sh so that |x| 2^-sh stays below 2^127.
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
    const float lo = __uint2float_rn(rem) * __int_as_float((fe - 52) << 23);   // rem 2^(fe-179)
    return {__int_as_float((int)hib), __int_as_float(__float_as_int(lo) | (int)sign)};
}

// a * b with a, b as (hi, lo): hi*hi exactly as p + e (FMA), plus the cross terms.
__device__ __forceinline__ f2 df_mul(f2 a, f2 b)
{
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return {p, e + fmaf(a.hi, b.lo, a.lo * b.hi)};
}

__device__ __forceinline__ f2 df_sqr(f2 a)
{
    const float p = a.hi * a.hi;
    const float e = fmaf(a.hi, a.hi, -p);
    return {p, fmaf(2.0f * a.hi, a.lo, e)};
}

// s += x with Knuth's two-sum on the high parts; low parts and the rounding error are
// collected in s.lo.
__device__ __forceinline__ void df_acc(f2& s, f2 x)
{
    const float t = s.hi + x.hi;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (x.hi - bp);
    s.hi = t;
    s.lo += err + x.lo;
}

__device__ __forceinline__ f2 df_add(f2 a, f2 b)
{
    f2 s = a;
    df_acc(s, b);
    return s;
}

__device__ __forceinline__ double df_to_double(f2 a) { return (double)a.hi + (double)a.lo; }

}  // namespace mbh

// Device code of the mixed-precision (float32-ratio) path, shared by the kernels of
// mbh_mixed.cu and by the extended-precision heterodyne (mbh_hetx.cu), which takes the float32
// edge ratio on edges of small contraction weight.  The large phase Phi(f) = Psi(f) +
// 2 pi f k.c(t(f)) (up to ~1e7 rad) is carried in double-float; amplitudes, the response and
// the ratio are float32 (see mbh_mixed.cu for the design notes).
#pragma once
#include <cuda_runtime.h>

#include "mbh_df.cuh"
#include "mbh_internal.cuh"
#include "mbh_model.cuh"

namespace mbh {

struct cf { float re, im; };
__device__ __forceinline__ cf fmul(cf a, cf b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf fadd(cf a, cf b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf fsub(cf a, cf b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cf fscale(cf a, float s) { return {a.re * s, a.im * s}; }

// float32 copies of the response constants of a walker
struct WalkerF {
    // k/sqrt3; the polarisation basis u/sqrt3, v/sqrt3 (e+ = uu - vv, ex = uv + vu); the mode
    // factors rotated by the polarisation angle, Ga = cos2psi K+ - sin2psi Kx and
    // Gb = sin2psi K+ + cos2psi Kx, so that n.P+.n K+ + n.Px.n Kx = a Ga + b Gb with
    // a = (u.n)^2 - (v.n)^2, b = 2 (u.n)(v.n); Glo: the float32 rounding of Ga, Gb (float pairs)
    float k[3], eu[3], ev[3], Ga[2], Gb[2], Glo[4];
    float eulo[2], evlo[3];   // the float32 rounding of eu (eu[2] = 0) and ev: float pairs
    float sa_ref, ca_ref, amp, inv_fc2;
    float amp76;   // amp (pi M)^{-7/6}: times f^{-7/6} of an edge table gives amp v^{-7/2}
    // relative rounding errors (exact/float - 1) of amp and amp76: a pure scale of the whole
    // template, which the heterodyne kernels undo exactly at the end (amp_fix)
    float eps_amp, eps_amp76;
};


// sin x / x as its Taylor series in u2 = x^2 to the term x^{2(N-1)}/(2N-1)!
template <int N>
__device__ __forceinline__ float sinc_series(float u2)
{
    // (-1)^j/(2j+1)!, j = 0..7
    constexpr float c[8] = {1.0f, -1.0f / 6.0f, 1.0f / 120.0f, -1.0f / 5040.0f, 1.0f / 362880.0f,
                            -1.0f / 39916800.0f, 1.0f / 6227020800.0f, -1.0f / 1307674368000.0f};
    float p = c[N - 1];
#pragma unroll
    for (int j = N - 2; j >= 0; --j) p = fmaf(p, u2, c[j]);
    return p;
}

// sin x / x: the series to x^14/15! for |x| < 2 (truncation < 2e-10), else sinf/x.
__device__ __forceinline__ float sincf(float x)
{
    if (fabsf(x) >= 2.0f) return sinf(x) / x;
    return sinc_series<8>(x * x);
}

// sin and cos of |r| <= pi/4 without reduction: Taylor polynomials of sin to r^9/9! and cos to
// r^10/10! (truncation < 2e-9), or with kShort (|r| <= 0.06) to r^5/5! and r^6/6! (< 1e-12)
template <bool kShort>
__device__ __forceinline__ void sincos_poly(float r, float* s, float* c)
{
    const float r2 = r * r;
    if (kShort) {
        *s = fmaf(fmaf(r2, 1.0f / 120.0f, -1.0f / 6.0f) * r2, r, r);
        *c = fmaf(fmaf(fmaf(r2, -1.0f / 720.0f, 1.0f / 24.0f), r2, -0.5f), r2, 1.0f);
        return;
    }
    float sp = fmaf(r2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    sp = fmaf(sp, r2, 1.0f / 120.0f);
    sp = fmaf(sp, r2, -1.0f / 6.0f);
    *s = fmaf(sp * r2, r, r);
    float cp = fmaf(r2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    cp = fmaf(cp, r2, -1.0f / 720.0f);
    cp = fmaf(cp, r2, 1.0f / 24.0f);
    cp = fmaf(cp, r2, -0.5f);
    *c = fmaf(cp, r2, 1.0f);
}

// sin and cos of |x| <~ 100: Cody-Waite reduction by pi/2 (two-term split of pi/2, the first
// product exact inside the FMA), then the Taylor polynomials of sin (to r^9/9!) and cos (to
// r^10/10!) on |r| <= pi/4 (truncation < 2e-9), rotated by the quadrant.
__device__ __forceinline__ void sincos_small(float x, float* s, float* c)
{
    const float q = rintf(x * 0.636619772f);                 // 2/pi
    float r = fmaf(-q, 1.57079637f, x);                       // float(pi/2)
    r = fmaf(-q, -4.37113883e-8f, r);                         // pi/2 - float(pi/2)
    const float r2 = r * r;
    float sp = fmaf(r2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    sp = fmaf(sp, r2, 1.0f / 120.0f);
    sp = fmaf(sp, r2, -1.0f / 6.0f);
    const float sr = fmaf(sp * r2, r, r);
    float cp = fmaf(r2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    cp = fmaf(cp, r2, -1.0f / 720.0f);
    cp = fmaf(cp, r2, 1.0f / 24.0f);
    cp = fmaf(cp, r2, -0.5f);
    const float cr = fmaf(cp, r2, 1.0f);
    const int iq = (int)q;
    const bool swap = iq & 1;
    const float s0 = swap ? cr : sr, c0 = swap ? sr : cr;
    *s = (iq & 2) ? -s0 : s0;
    *c = ((iq + 1) & 2) ? -c0 : c0;
}

// sinc(x (1 + k)) - sinc(x (1 - k)) without cancellation: for arguments below 2 as
// (a^2 - b^2) sum_{j>=1} (-1)^j P_j / (2j+1)!, P_1 = 1, P_{j+1} = a^2 P_j + b^{2j}
// (a^{2j} - b^{2j} = (a^2 - b^2) P_j), with a^2 - b^2 = 4 x^2 k; directly above.
// the series of sinc(x(1 + k)) - sinc(x(1 - k)) with N terms (j = 1..N)
template <int N>
__device__ __forceinline__ float sinc_diff_series(float x, float k)
{
    const float a = x * (1.0f + k), b = x * (1.0f - k);
    const float a2 = a * a, b2 = b * b;
    // 1/(2j+1)! for j = 1..9 (terms beyond are below 5e-12 relative for arguments < 2)
    constexpr float inv_fact[9] = {1.0f / 6.0f, 1.0f / 120.0f, 1.0f / 5040.0f, 1.0f / 362880.0f,
                                   1.0f / 39916800.0f, 1.0f / 6227020800.0f, 1.0f / 1307674368000.0f,
                                   1.0f / 355687428096000.0f, 1.0f / 121645100408832000.0f};
    float P = 1.0f, bp = 1.0f, sum = 0.0f, sign = -1.0f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        sum += sign * P * inv_fact[j];
        sign = -sign;
        bp *= b2;
        P = a2 * P + bp;
    }
    return 4.0f * x * x * k * sum;
}

__device__ __forceinline__ float sinc_diff(float x, float k)
{
    const float a = x * (1.0f + k), b = x * (1.0f - k);
    if (fmaxf(fabsf(a), fabsf(b)) >= 2.0f) return sincf(a) - sincf(b);
    return sinc_diff_series<9>(x, k);
}

// Below x = 0.1 (both arguments under 0.2, |k| <= 1) four terms of either series reach float32
// rounding (the next terms are below 1e-11 and 3e-13 of the first): the short forms used there.
constexpr float kSincShortX = 0.1f;

// Transfer T_c(f) in float32, times a real factor `scale` (the caller's amplitude): the
// construction of transfer_f64, rearranged so that no step cancels to leading order at small
// f L (which float32 cannot afford):
//   1 - D = 2i sin x e^{-ix}, 1 - D^2 = 2i sin 2x e^{-2ix} (no 1 - cos), and
//   X + Y + Z = (1 - D^2)(1 - D) sum_arms g_a [sinc(x(1 + k.n)) - sinc(x(1 - k.n))],
// so T = (X + Y + Z)/sqrt3 is formed from sinc differences computed without cancellation.
// Spacecraft offsets from the guiding centre are u_i L/sqrt3 (|u_i - u_j| = sqrt3,
// u_0 + u_1 + u_2 = 0); the walker carries k/sqrt3 and P/3 (WalkerF), so with
// kappa_m = (k/sqrt3).u_m: k.n = kappa_j - kappa_i and n.P.n = (u_j - u_i).(P/3).(u_j - u_i) on
// the arm from i to j, whose one-link phase pi f (L + k.(p_i + p_j)) is x - q_m, q_m = x kappa_m
// for the third spacecraft m (q_0 + q_1 + q_2 = 0, |q_m| <= x/sqrt3): e^{i q_m} for m = 0, 1
// from their polynomials, the third the conjugate of their product.  Common factors (1 - D^2,
// the one-link -x, e^{-ix}, scale and the A/E/T normalisations) multiply once at the end:
//   X = (1 - D^2) [(y21 - y31) + D (y12 - y13)] and cyclic.
// With kRaw every factor that depends on the frequency alone is left out (and `scale` is not
// applied): T_A = Z' - X', T_E = X' + Z' - 2Y', T_T = sum_arms g_a [sinc differences] with
// X' = X/(1 - D^2) etc.  The heterodyne folds the rest, per edge and channel, into its
// float64-formed 1/h0 (so that no float32 rounding of a per-edge or constant factor is shared
// by every walker's template, which would bias the whole batch).
// Ga, Gb: the walker's rotated mode factors (WalkerF, or a higher mode's); Glo (or nullptr):
// their low parts as float pairs (Ga_lo[2], Gb_lo[2]).
template <bool kRaw = false>
__device__ inline void transfer_f32(const WalkerF& w, const float* Ga, const float* Gb, float x, float sa,
                                    float ca, float scale, float s1, float c1, cf T[3],
                                    const float* Glo = nullptr)
{
    // sqrt3/2 as a float pair: its float32 rounding alone would shorten the arms by ~2e-8 for
    // every walker alike (a bias of the whole batch)
    constexpr float h3 = (float)(0.5 * kSqrt3);
    constexpr float h3lo = (float)(0.5 * kSqrt3 - (double)h3);
    const float h3s = fmaf(h3, sa, h3lo * sa), h3c = fmaf(h3, ca, h3lo * ca);
    const float sp[3] = {sa, -0.5f * sa - h3c, -0.5f * sa + h3c};
    const float cp[3] = {ca, -0.5f * ca + h3s, -0.5f * ca - h3s};
    float u[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        u[i][0] = -sp[i] * sa - 0.5f * cp[i] * ca;
        u[i][1] = sp[i] * ca - 0.5f * cp[i] * sa;
        u[i][2] = -fmaf(h3, cp[i], h3lo * cp[i]);
    }
    float kap[3];
#pragma unroll
    for (int m = 0; m < 2; ++m) kap[m] = w.k[0] * u[m][0] + w.k[1] * u[m][1] + w.k[2] * u[m][2];
    kap[2] = -(kap[0] + kap[1]);
    const bool shrt = x < kSincShortX;   // uniform over a warp but for the rounds that straddle 0.1
    cf E[3];                             // e^{i q_m}
    if (shrt) {
        sincos_poly<true>(x * kap[0], &E[0].im, &E[0].re);
        sincos_poly<true>(x * kap[1], &E[1].im, &E[1].re);
    } else if (x < 1.36f) {              // |q_m| <= x/sqrt3 < pi/4
        sincos_poly<false>(x * kap[0], &E[0].im, &E[0].re);
        sincos_poly<false>(x * kap[1], &E[1].im, &E[1].re);
    } else {
        sincos_small(x * kap[0], &E[0].im, &E[0].re);
        sincos_small(x * kap[1], &E[1].im, &E[1].re);
    }
    const cf e01 = fmul(E[0], E[1]);
    E[2] = {e01.re, -e01.im};
    cf yf[3], yb[3], tsum = {0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = a, j = (a + 1) % 3, m = (a + 2) % 3;
        float d[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] = u[j][q] - u[i][q];
        const float kn = kap[j] - kap[i];
        // n.P+.n K+ + n.Px.n Kx = a Ga + b Gb (n = d/sqrt3; eu, ev carry the 1/sqrt3)
        // (u, v as float pairs: their rounding would otherwise be common to every edge)
        const float un = fmaf(w.eu[0], d[0], fmaf(w.eu[1], d[1], w.eulo[0] * d[0] + w.eulo[1] * d[1]));
        const float vn = fmaf(w.ev[0], d[0], fmaf(w.ev[1], d[1], fmaf(w.ev[2], d[2],
                              w.evlo[0] * d[0] + w.evlo[1] * d[1] + w.evlo[2] * d[2])));
        const float pa = fmaf(un, un, -vn * vn), pb = 2.0f * un * vn;
        cf F = {pa * Ga[0] + pb * Gb[0], pa * Ga[1] + pb * Gb[1]};
        if (Glo != nullptr) {   // the factors' float32 rounding is common to all edges
            F.re += pa * Glo[0] + pb * Glo[2];
            F.im += pa * Glo[1] + pb * Glo[3];
        }
        const cf g = fmul({-E[m].im, E[m].re}, F);   // i e^{i q_m} F
        // sinc(x(1 + k.n)) = sinc(x(1 - k.n)) + the difference (which T needs on its own);
        // the sum is off by at most an ulp of the larger term, like a direct evaluation
        float sm, sd;
        if (shrt) {
            const float b = x * (1.0f - kn);
            sm = sinc_series<4>(b * b);
            sd = sinc_diff_series<4>(x, kn);
        } else {
            sm = sincf(x * (1.0f - kn));
            sd = sinc_diff(x, kn);
        }
        yf[a] = fscale(g, sm);
        yb[a] = fscale(g, sm + sd);
        tsum = fadd(tsum, fscale(g, sd));   // y_{j->i} - y_{i->j}
    }
    const cf y12 = yf[0], y21 = yb[0], y23 = yf[1], y32 = yb[1], y31 = yf[2], y13 = yb[2];
    const float s2 = 2.0f * s1 * c1, c2 = 1.0f - 2.0f * s1 * s1;   // sin 2x, cos 2x
    const cf D = {c2, -s2};
    const cf Xp = fadd(fsub(y21, y31), fmul(D, fsub(y12, y13)));
    const cf Yp = fadd(fsub(y32, y12), fmul(D, fsub(y23, y21)));
    const cf Zp = fadd(fsub(y13, y23), fmul(D, fsub(y31, y32)));
    if (kRaw) {
        T[0] = fsub(Zp, Xp);
        T[1] = fsub(fadd(Xp, Zp), fscale(Yp, 2.0f));
        T[2] = tsum;
    } else {
        const cf W1 = {2.0f * s1 * s1, 2.0f * s1 * c1};   // 1 - D
        // (1 - D^2) (-x) e^{-ix} scale = -2 x scale sin 2x (sin 3x, cos 3x)
        const float w2 = -x * scale * 2.0f * s2;
        const cf W2 = {w2 * (s2 * c1 + c2 * s1), w2 * (c2 * c1 - s2 * s1)};
        T[0] = fmul(fscale(W2, (float)(1.0 / kSqrt2)), fsub(Zp, Xp));
        T[1] = fmul(fscale(W2, (float)(1.0 / kSqrt6)), fsub(fadd(Xp, Zp), fscale(Yp, 2.0f)));
        T[2] = fmul(fscale(fmul(W2, W1), (float)(1.0 / kSqrt3)), tsum);
    }
}

// the same with sin x, cos x of the one-link phase x = pi f L/c computed here
__device__ __forceinline__ void transfer_f32(const WalkerF& w, const float* Ga, const float* Gb, float f,
                                             float sa, float ca, float scale, cf T[3])
{
    const float x = (float)kPi * (float)kArmSec * f;
    float s1, c1;
    sincos_small(x, &s1, &c1);
    transfer_f32<false>(w, Ga, Gb, x, sa, ca, scale, s1, c1, T);
}

constexpr f2 kTwoPiDF = df_const(kTwoPi);

// Per-walker constants of the phase chain as float pairs.
struct WalkerDF {
    f2 c[8], d[8], cl5, cl6, dl6;
    f2 cbrt_piM, icbrt_piM, ln_cbrt_piM;
    f2 tref, fcut, t0, c1;
    f2 sa_ref, ca_ref, kx, ky;
};

__device__ __forceinline__ f2 split_d(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// v and ln v at f_max: pi M f_max = 0.05 pi sqrt(5/12) = 0.1013944668993403 for every mass
// (f_max = f_c sqrt(5/12), f_c = 0.05/M), so v(f_max) = (pi M f_max)^{1/3}, ln v(f_max), v^-5
// and v^-8 are constants (evaluated to 40 digits, then rounded).
constexpr double kVm = 0.4663064457284195;
constexpr double kLnVm = -0.7629122521271803;
constexpr double kVmPow5Inv = 45.35685218040481;
constexpr double kVmPow8Inv = 447.3306440422728;

// float64 values of constants that WalkerDF carries as float pairs, for callers that need
// them beyond the pairs' ~48 bits (the extended direct pass)
struct WalkerDFFull {
    double c1, c0, icb;   // c1; c_0 (the 0PN phase coefficient); (pi M)^{-1/3}
};

// Per-walker constants of the mixed path (Sec. II A parameter derivation), in float64: the
// large-phase constants (PN coefficients, the v and ln v scales, t_ref and the f_max
// references, the orbital angle at t_ref, the in-plane propagation components) are split
// into float pairs with integer operations (split_f64); the amplitude, polarisation and mode
// factors are rounded once to float32.  One thread per walker; the caller spreads walkers
// over full warps (a float64 warp instruction costs the same with 4 or 32 active lanes).
__device__ inline void walker_setup_mixed(const double* __restrict__ theta, int64_t W, int64_t i,
                                          WalkerDF& m, WalkerF& wf, WalkerDFFull* full = nullptr)
{
    const double mt = theta[kMT * W + i], q = theta[kQ * W + i];
    const double a1 = theta[kA1 * W + i], a2 = theta[kA2 * W + i];
    const double tref = theta[kTref * W + i];
    const double lam = theta[kLam * W + i], bet = theta[kBeta * W + i];
    const double dl = theta[kDL * W + i], phi = theta[kPhi * W + i];
    const double iota = theta[kIota * W + i], pol = theta[kPsi * W + i];

    // few float64 divisions and transcendentals: on this path they cost 16 cycles of the SM's
    // float64 pipe per warp instruction, and the setup runs in every block before its edges
    // one float64 division for four reciprocals: 1/(1+q), 1/q, 1/M and 1/D from 1/((1+q) q M D)
    const double opq = 1.0 + q;
    const double M = mt * kMsunSec;
    const double dist = (double)dl * (1e9 * kParsec / kClight);
    const double qM = q * M, od = opq * dist;
    const double rr = 1.0 / (qM * od);
    const double x1 = rr * qM * dist, iq = rr * M * od, iM = rr * q * od, idist = rr * qM * opq;
    const double x2 = q * x1;
    const double eta = x1 * x2;
    const double so = (113.0 / 12.0 * x1 * x1 + 25.0 / 4.0 * eta) * a1 +
                      (113.0 / 12.0 * x2 * x2 + 25.0 / 4.0 * eta) * a2;
    const double ss = 79.0 / 8.0 * eta * a1 * a2;
    const double pi2 = kPi * kPi;
    double al[8];
    al[0] = 1.0;
    al[1] = 0.0;
    al[2] = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
    al[3] = -16.0 * kPi + 4.0 * so;
    al[4] = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta - 10.0 * ss;
    al[5] = kPi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
    const double alog5 = 3.0 * al[5];
    al[6] = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi2 - 6848.0 / 21.0 * kEulerGamma -
            6848.0 / 21.0 * 1.386294361119890618834464242916353136 +
            eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2) + 76055.0 / 1728.0 * eta * eta -
            127825.0 / 1296.0 * eta * eta * eta;
    const double alog6 = -6848.0 / 21.0;
    al[7] = kPi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta);
    const double pre = (3.0 / 128.0) * opq * opq * iq, dpre = pre * (kPi / 3.0) * M;   // 3/(128 eta)
    double c[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        c[k] = pre * al[k];
        d[k] = dpre * ((k - 5) * al[k]);
    }
    d[5] += dpre * alog5;
    d[6] += dpre * alog6;
    const double cl5 = pre * alog5, cl6 = pre * alog6, dl6 = dpre * alog6;
    // Psi_PN and its derivative at f_max (v = constant)
    double P = c[7], Q = d[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        P = fma(P, kVm, c[k]);
        Q = fma(Q, kVm, d[k]);
    }
    constexpr double vm5 = kVm * kVm * kVm * kVm * kVm, vm6 = vm5 * kVm;
    const double psi_max = (P + kLnVm * (cl5 * vm5 + cl6 * vm6)) * kVmPow5Inv;
    const double dpsi_max = (Q + kLnVm * dl6 * vm6) * kVmPow8Inv;
    const double piM = kPi * M;
    const double icb = rcbrt(piM), cb = piM * icb * icb;
    double sa, ca, sl, cl, sb, cbt;
    sincos(kTwoPi * tref / kYear, &sa, &ca);
    sincos(lam, &sl, &cl);
    sincos(bet, &sb, &cbt);
    // Phi(f) = f (c1 + ...) + Psi_PN(f) + c0 (the pinning below): c0 joins the constant term c_5
    const double fmax = (0.05 * 0.6454972243679028) * iM;   // f_c sqrt(5/12)
    const double c0 = fmax * dpsi_max - psi_max;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        m.c[k] = split_f64(k == 5 ? c[5] + c0 : c[k], 0);
        m.d[k] = split_f64(d[k] * kInvTwoPi, 0);   // the derivative chain gives t(f) in seconds
    }
    m.cl5 = split_f64(cl5, 0);
    m.cl6 = split_f64(cl6, 0);
    m.dl6 = split_f64(dl6 * kInvTwoPi, 0);
    m.cbrt_piM = split_f64(cb, 0);
    m.icbrt_piM = split_f64(icb, 0);
    m.ln_cbrt_piM = split_f64(log(piM) * (1.0 / 3.0), 0);
    // the t_ref and f_max pinning folded into per-walker constants:
    //   t(f) = t_ref + (Psi'(f) - Psi'(f_max))/(2 pi) = Psi'(f)/(2 pi) + t0,
    //   Phi(f) = 2 pi f (t_ref + k.c(t)) + Psi_PN(f) - Psi_PN(f_max) - (f - f_max) Psi'(f_max)
    //          = f (c1 + 2 pi (AU/c) k.(c(t) - c(t_ref))) + Psi_PN(f) + c0
    m.tref = split_f64(tref, 0);
    m.fcut = split_d(0.2 * iM);   // rounded to nearest: compared lexicographically (dd_le)
    m.t0 = split_f64(tref - dpsi_max * kInvTwoPi, 0);
    const double kxd = kTwoPi * kAUSec * (-cbt * cl), kyd = kTwoPi * kAUSec * (-cbt * sl);
    const double c1d = kTwoPi * tref - dpsi_max + (kxd * ca + kyd * sa);   // with k.c(t_ref)
    m.c1 = split_f64(c1d, 0);
    if (full) {
        full->c1 = c1d;
        full->c0 = c[0];
        full->icb = icb;
    }
    m.sa_ref = split_d(sa);   // high parts rounded to nearest (the orbit's sin, cos per point)
    m.ca_ref = split_d(ca);
    m.kx = split_f64(kxd, 0);
    m.ky = split_f64(kyd, 0);

    // Float32 constants (amplitude, taper, wave frame, mode factors), computed in float64 and
    // rounded once: the heterodyne ratio h/h0 of a nearby walker cancels their common part,
    // so their rounding error enters the likelihood directly.
    // A = sqrt(2 pi/3) pi^{-2/3} M^{5/6} eta^{1/2} (pi M)^{7/6} / D v^{-7/2} exp(-(f/fc)^2)
    //   = pi sqrt(2/3) M^2 sqrt(eta) / D v^{-7/2} exp(-(f/fc)^2)
    const double ampd = kPi * 0.816496580927726 /* sqrt(2/3) */ * M * M * sqrt(eta) * idist;
    const double amp76d = ampd * (icb * icb * icb) * sqrt(icb);   // (pi M)^{-7/6} = icb^{7/2}
    wf.amp = (float)ampd;
    wf.amp76 = (float)amp76d;
    wf.eps_amp = (float)(ampd - (double)wf.amp) / wf.amp;
    wf.eps_amp76 = (float)(amp76d - (double)wf.amp76) / wf.amp76;
    wf.inv_fc2 = (float)(400.0 * M * M);   // 1/f_c^2, f_c = 0.05/M
    wf.sa_ref = (float)sa;
    wf.ca_ref = (float)ca;
    double s2p, c2p, s2f, c2f;
    sincos(2.0 * (double)pol, &s2p, &c2p);
    sincos(2.0 * (double)phi, &s2f, &c2f);
    // k, u, v over sqrt3 (the response works with spacecraft offsets in units of L/sqrt3)
    constexpr double isq3 = 0.57735026918962576;
    wf.k[0] = (float)(-cbt * cl * isq3);
    wf.k[1] = (float)(-cbt * sl * isq3);
    wf.k[2] = (float)(-sb * isq3);
    const double eu[2] = {sl * isq3, -cl * isq3};
    const double ev[3] = {-sb * cl * isq3, -sb * sl * isq3, cbt * isq3};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        wf.eu[j] = j < 2 ? (float)eu[j] : 0.0f;
        wf.ev[j] = (float)ev[j];
        wf.evlo[j] = (float)(ev[j] - (double)wf.ev[j]);
        if (j < 2) wf.eulo[j] = (float)(eu[j] - (double)wf.eu[j]);
    }
    const double ylm = 0.15769578262626002 /* sqrt(5/(64 pi)) */;
    const double ci = cos((double)iota);
    const double ap = ylm * (1.0 + ci * ci), ac = 2.0 * ylm * ci;
    // K+ = ap e^{2i phi}, Kx = i ac e^{2i phi}; Ga = cos2psi K+ - sin2psi Kx, Gb = sin2psi K+ + cos2psi Kx
    const double g[4] = {c2p * ap * c2f + s2p * ac * s2f, c2p * ap * s2f - s2p * ac * c2f,
                         s2p * ap * c2f - c2p * ac * s2f, s2p * ap * s2f + c2p * ac * c2f};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        wf.Ga[j] = (float)g[j];
        wf.Gb[j] = (float)g[2 + j];
        wf.Glo[j] = (float)(g[j] - (double)wf.Ga[j]);
        wf.Glo[2 + j] = (float)(g[2 + j] - (double)wf.Gb[j]);
    }
}

// The float32 amplitude factors of the walker and of the reference scale the whole of h and h0,
// so their rounding is a common factor of every ratio r = h/h0: <d|h> (linear in r) is off by
// amp_fix and <h|h> (quadratic) by its square, which the epilogue removes in float64.  Left in,
// this coherent error dominates |dlnL| for walkers far from the reference.
__device__ __forceinline__ double amp_fix(float eps_walker, double eps_ref)
{
    return (1.0 + (double)eps_walker) / (1.0 + eps_ref);
}

// frequency tables of one grid point: f, f^{1/3}, f^{-1/3}, ln(f)/3 as float pairs
struct FreqDF {
    f2 f, f3, fm3, lnf3;
};

__device__ __forceinline__ FreqDF freq_tables(double f)
{
    const double f3 = cbrt(f);
    return {split_d(f), split_d(f3), split_d(1.0 / f3), split_d(log(f) * (1.0 / 3.0))};
}

__device__ __forceinline__ f2 ld_f2(float2 v) { return {v.x, v.y}; }

// Large phase Phi(f) (double-float) and float32 amplitude and orbit angle from the
// frequency tables.  Returns false outside the support (f > f_cut or t(f) outside [0, t_obs]);
// with kAlways the phase is computed there as well (a reference phase defined at every edge).
// With kTab the amplitude leaves out f^{-7/6} (amp76 e^{-(f/f_c)^2}), which the heterodyne folds
// into its edge records.
template <bool kAlways = false, bool kTab = false>
__device__ __forceinline__ bool phase_df(const WalkerDF& w, const WalkerF& wf, const FreqDF& q,
                                         f2 t_obs, f2& Phi, float& sa, float& ca, float& amp)
{
    // intermediate double-float values stay unnormalised (the *_lazy forms) up to the two that
    // need it: t(f), compared against the support bounds, and Phi
    const f2 v = dd_mul_lazy(w.cbrt_piM, q.f3);
    const f2 iv = dd_mul_lazy(w.icbrt_piM, q.fm3);
    const f2 lnv = dd_add_lazy(w.ln_cbrt_piM, q.lnf3);
    // Psi_PN = sum_k c_k v^{k-5} + ln v (cl5 + cl6 v): the powers v^-5..v^0 by Horner in 1/v
    // (c_1 = 0, no 0.5PN term: the first step is the product c_0 / v), v and v^2 by Horner in v
    f2 N = dd_mul_lazy(w.c[0], iv);
#pragma unroll
    for (int k = 2; k <= 5; ++k) N = dd_fma_lazy(N, iv, w.c[k]);
    const f2 Pp = dd_mul_lazy(dd_fma_lazy(w.c[7], v, w.c[6]), v);
    const f2 psi_pn = dd_add_lazy(dd_add_lazy(N, Pp), dd_mul_lazy(lnv, dd_fma_lazy(w.cl6, v, w.cl5)));
    // t(f) = Psi'(f)/(2 pi) + t0 (the walker's d and dl6 carry the 1/(2 pi))
    float dt;   // t - t_ref
    bool in;
    if (kAlways) {
        const f2 iv2 = dd_mul_lazy(iv, iv), iv4 = dd_mul_lazy(iv2, iv2), iv8 = dd_mul_lazy(iv4, iv4);
        f2 Q = w.d[7];
#pragma unroll
        for (int k = 6; k >= 0; --k) Q = dd_fma_lazy(Q, v, w.d[k]);
        const f2 t = dd_add(dd_add_lazy(dd_mul_lazy(Q, iv8), dd_mul_lazy(dd_mul_lazy(lnv, w.dl6), iv2)), w.t0);
        in = dd_le(q.f, w.fcut) && !dd_lt0(t) && dd_le(t, t_obs);
        dt = __fadd_rn(__fsub_rn(t.hi, w.tref.hi), __fsub_rn(t.lo, w.tref.lo));
    } else {
        // t - t_ref in float32: it only turns the orbit (an error of 1e-6 |t - t_ref| moves
        // the SSB delay phase by < 1e-7 rad at every frequency of the band), and the support
        // test t in [0, t_obs] takes the double-float t only where the float32 value's error
        // bound straddles a bound (rounding of the Horner sum, the float32 powers of v and ln v:
        // < 3e-6 of the sum of |terms|; bound 1e-5)
        const float vf = v.hi, i2 = iv.hi * iv.hi, i4 = i2 * i2, i8 = i4 * i4;
        float Qf = w.d[7].hi, Qa = fabsf(w.d[7].hi);
#pragma unroll
        for (int k = 6; k >= 0; --k) {
            Qf = fmaf(Qf, vf, w.d[k].hi);
            Qa = fmaf(Qa, vf, fabsf(w.d[k].hi));
        }
        const float t2 = lnv.hi * w.dl6.hi * i2;
        const float dtc = __fadd_rn(__fsub_rn(w.t0.hi, w.tref.hi), __fsub_rn(w.t0.lo, w.tref.lo));
        dt = fmaf(Qf, i8, t2) + dtc;
        const float lo = (dt + w.tref.hi) + w.tref.lo;                          // t
        const float hi = (dt + (w.tref.hi - t_obs.hi)) + (w.tref.lo - t_obs.lo);   // t - t_obs
        const float err = 1e-5f * fmaf(Qa, i8, fabsf(t2)) + 3e-7f * (fabsf(dtc) + fabsf(lo) + fabsf(hi)) + 1e-6f;
        in = dd_le(q.f, w.fcut);
        if (lo >= err && hi <= -err) {
            // inside
        } else if (lo < -err || hi > err) {
            in = false;
        } else {   // within the bound of t = 0 or t = t_obs: the double-float t decides
            const f2 iv2 = dd_mul_lazy(iv, iv), iv4 = dd_mul_lazy(iv2, iv2), iv8 = dd_mul_lazy(iv4, iv4);
            f2 Q = w.d[7];
#pragma unroll
            for (int k = 6; k >= 0; --k) Q = dd_fma_lazy(Q, v, w.d[k]);
            const f2 t = dd_add(dd_add_lazy(dd_mul_lazy(Q, iv8), dd_mul_lazy(dd_mul_lazy(lnv, w.dl6), iv2)), w.t0);
            in = in && !dd_lt0(t) && dd_le(t, t_obs);
        }
        if (!in) return false;
    }
    const float da = dt * (float)(kTwoPi / kYear);
    float sh, ch;
    sincos_small(0.5f * da, &sh, &ch);
    const float sd = 2.0f * sh * ch, omc = 2.0f * sh * sh;   // sin da, 1 - cos da
    const float ds = wf.ca_ref * sd - wf.sa_ref * omc;      // sin alpha - sin alpha(t_ref)
    const float dc = -(wf.ca_ref * omc + wf.sa_ref * sd);   // cos alpha - cos alpha(t_ref)
    // Phi = f (c1 + 2 pi (AU/c) k.c(t)) + Psi_PN(f) + c0 (kx, ky carry 2 pi AU/c); the walker's
    // c1 holds k.c(t_ref), so only the orbit's change since t_ref is added here, in float32
    // (its rounding, <= 1.2e-7 of f |k| |c(t) - c(t_ref)|, is below 1e-7 rad at every edge)
    const float dk = fmaf(w.kx.hi, dc, fmaf(w.ky.hi, ds, fmaf(w.kx.lo, dc, w.ky.lo * ds)));
    const f2 s1 = two_sum(w.c1.hi, dk);
    const f2 S = {s1.hi, __fadd_rn(s1.lo, w.c1.lo)};   // unnormalised operand of dd_mul_lazy
    Phi = dd_add(dd_mul_lazy(q.f, S), psi_pn);   // c0 is in the walker's c_5
    // sin, cos of the orbit angle: the reference's value rounded to nearest plus (the change
    // since t_ref plus that rounding).  Near the merger, where the edges carry the weight, the
    // change is small and the inner sum exact to far below an ulp of the result, so the one
    // rounding left is unbiased; a rounding of the reference's value alone would be common to
    // those edges (with a truncated high part, p99 |dlnL| 6e-4 -> 1.2e-3)
    sa = __fadd_rn(w.sa_ref.hi, __fadd_rn(ds, w.sa_ref.lo));
    ca = __fadd_rn(w.ca_ref.hi, __fadd_rn(dc, w.ca_ref.lo));
    const float ff = q.f.hi;
    if (kTab) {   // f^{-7/6} is folded into the edge table's 1/h0
        amp = wf.amp76 * expf(-ff * ff * wf.inv_fc2);
    } else {
        const float ivf = iv.hi;
        amp = wf.amp * ivf * ivf * ivf * sqrtf(ivf) * expf(-ff * ff * wf.inv_fc2);
    }
    return in;
}

// ---- higher harmonics, mixed precision ---------------------------------------------------
// Mode (l, m) is the (2,2) chain at f2 = 2f/m (so its tables are the grid's scaled by
// constants) with the phase scaled by m/2; the amplitude gains v^{p_lm} and the response uses
// the mode's polarisation factors (float32, folded with H_lm's constant and sqrt(2/m)).
struct WalkerHMF {
    float hk[kHmModes][4];     // per mode Ga (re, im), Gb (re, im), as WalkerF's for the (2,2) mode
    float hklo[kHmModes][4];   // their float32 rounding (float pairs)
};

// tables of f2 = r f, r = 2/m: f2, f2^{1/3}, f2^{-1/3}, ln(f2)/3
__device__ __forceinline__ FreqDF mode_tables(const FreqDF& q, int b)
{
    constexpr f2 r[kHmModes] = {df_const(1.0), df_const(2.0 / 3.0), df_const(0.5), df_const(2.0),
                                df_const(1.0), df_const(2.0 / 3.0)};
    constexpr f2 r3[kHmModes] = {df_const(1.0), df_const(0.87358046473629952), df_const(0.79370052598409974),
                                 df_const(1.2599210498948732), df_const(1.0), df_const(0.87358046473629952)};
    constexpr f2 rm3[kHmModes] = {df_const(1.0), df_const(1.1447142425533319), df_const(1.2599210498948732),
                                  df_const(0.79370052598409974), df_const(1.0), df_const(1.1447142425533319)};
    constexpr f2 ln3[kHmModes] = {df_const(0.0), df_const(-0.13515503603605479), df_const(-0.23104906018664842),
                                  df_const(0.23104906018664842), df_const(0.0), df_const(-0.13515503603605479)};
    if (hm_m(b) == 2) return q;
    return {dd_mul(q.f, r[b]), dd_mul(q.f3, r3[b]), dd_mul(q.fm3, rm3[b]), dd_add(q.lnf3, ln3[b])};
}

// Phi_lm = (m/2) Phi_22(f2) in double-float (exact for m = 1, 2, 4)
__device__ __forceinline__ f2 mode_phase(f2 p, int b)
{
    const int m = hm_m(b);
    if (m == 2) return p;
    if (m == 4) return {2.0f * p.hi, 2.0f * p.lo};
    if (m == 1) return {0.5f * p.hi, 0.5f * p.lo};
    return dd_mul_f(p, 1.5f);
}

// Folded per-mode factors of one walker (float64, rounded once), as in the float64 model.
__device__ inline void walker_setup_hm(const double* __restrict__ theta, int64_t W, int64_t i,
                                       WalkerHMF& h)
{
    const double q = theta[kQ * W + i], iota = theta[kIota * W + i], phi = theta[kPhi * W + i];
    const double pol = theta[kPsi * W + i];
    Walker tmp;
    hm_setup(tmp, q, iota, phi);
    double s2p, c2p;
    sincos(2.0 * pol, &s2p, &c2p);
    // per mode (Ga, Gb) = (cos2psi K+ - sin2psi Kx, sin2psi K+ + cos2psi Kx) as transfer_f32 takes them
#pragma unroll
    for (int b = 0; b < kHmModes; ++b)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double kp = tmp.hk[b][j], kc = tmp.hk[b][2 + j];
            const double ga = c2p * kp - s2p * kc, gb = s2p * kp + c2p * kc;
            h.hk[b][j] = (float)ga;
            h.hk[b][2 + j] = (float)gb;
            h.hklo[b][j] = (float)(ga - (double)h.hk[b][j]);
            h.hklo[b][2 + j] = (float)(gb - (double)h.hk[b][2 + j]);
        }
}

// modes (mask bits) of the four values of m: group 0 m = 2 ((2,2), (3,2)), 1 m = 3 ((3,3),
// (4,3)), 2 m = 4 ((4,4)), 3 m = 1 ((2,1))
__host__ __device__ constexpr uint32_t hm_group_mask(int grp)
{
    return grp == 0 ? 0x11u : grp == 1 ? 0x22u : grp == 2 ? 0x04u : 0x08u;
}

// v^{p_lm} in float32 from f2^{1/3} and (pi M)^{1/3}
__device__ __forceinline__ float mode_vpow(const WalkerDF& w, const FreqDF& q2, int b)
{
    const f2 vv = dd_mul_lazy(w.cbrt_piM, q2.f3);   // both parts: the high parts' rounding
    const float v = vv.hi + vv.lo;                     // would bias v^p for every edge alike
    const int p = hm_vpow(b);
    return p == 0 ? 1.0f : p == 1 ? v : p == 2 ? v * v : v * v * v;
}



// phase modulo 2 pi in double-float, then float32
__device__ __forceinline__ float reduce_phase(f2 p)
{
    // p - 2 pi n with 2 pi as a float pair (Cody-Waite): n is an integer of up to ~21 bits
    // (|p| <~ 1e7), so p_hi - n (2 pi)_hi is exact in one FMA (its result needs no bits below
    // 2^-21 and fits 24), and the low parts add the remaining ~1e-9 rad
    const float n = rintf(p.hi * (float)kInvTwoPi);
    const float r = fmaf(-n, kTwoPiDF.hi, p.hi);
    return r + fmaf(-n, kTwoPiDF.lo, p.lo);
}

// Raw mixed template at one grid point (without the frequency-only factors K_c, which the
// fused pass folds into its data): amp76 e^{-(f/f_c)^2} e^{-i Phi} T_raw, times `scale`; xs holds
// sin x, cos x and x of the point (ftab3).
__device__ __forceinline__ bool point_mixed_raw(const WalkerDF& w, const WalkerF& wf, const FreqDF& q,
                                                float4 xs, f2 t_obs, float scale, cf h[3])
{
    f2 Phi;
    float sa, ca, amp;
    if (!phase_df<false, true>(w, wf, q, t_obs, Phi, sa, ca, amp)) return false;
    float sp, cp;
    sincos_small(reduce_phase(Phi), &sp, &cp);
    cf T[3];
    transfer_f32<true>(wf, wf.Ga, wf.Gb, xs.w, sa, ca, 1.0f, xs.x, xs.y, T, wf.Glo);
    const float a = amp * scale;
    const cf e = {a * cp, -a * sp};
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = fmul(e, T[c]);
    return true;
}

// Mixed template at one grid point: h = amp e^{-i Phi} T (float32 result, times `scale`).
__device__ __forceinline__ bool point_mixed(const WalkerDF& w, const WalkerF& wf, const FreqDF& q,
                                            f2 t_obs, float scale, cf h[3])
{
    f2 Phi;
    float sa, ca, amp;
    if (!phase_df(w, wf, q, t_obs, Phi, sa, ca, amp)) return false;
    float sp, cp;
    sincos_small(reduce_phase(Phi), &sp, &cp);
    cf T[3];
    transfer_f32(wf, wf.Ga, wf.Gb, q.f.hi, sa, ca, amp * scale, T);
    const cf e = {cp, -sp};
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = fmul(e, T[c]);
    return true;
}

// Mixed template of the walker's modes at one grid point (times `scale`): per mode the (2,2)
// chain at f2, the phase scaled by m/2 and reduced modulo 2 pi in double-float, the response
// at t_lm with the mode's factors; summed.  Returns false when no mode is in its support.
__device__ __forceinline__ bool point_mixed_hm(const WalkerDF& w, const WalkerF& wf, const WalkerHMF& wh,
                                               const FreqDF& q, f2 t_obs, float scale, uint32_t modes,
                                               cf h[3])
{
    h[0] = h[1] = h[2] = {0.0f, 0.0f};
    bool any = false;
    // one phase chain and one response per distinct m (as het_mixed_hm_kernel)
    for (int grp = 0; grp < 4; ++grp) {
        const uint32_t gmask = modes & hm_group_mask(grp);
        if (!gmask) continue;
        const int b0 = __ffs(gmask) - 1;
        const FreqDF q2 = mode_tables(q, b0);
        f2 Phi;
        float sa, ca, amp;
        if (!phase_df(w, wf, q2, t_obs, Phi, sa, ca, amp)) continue;
        any = true;
        float sp, cp;
        sincos_small(reduce_phase(mode_phase(Phi, b0)), &sp, &cp);
        float gk[4] = {0.f, 0.f, 0.f, 0.f};
        for (uint32_t bm = gmask; bm; bm &= bm - 1) {
            const int b = __ffs(bm) - 1;
            const float vp = mode_vpow(w, q2, b);
#pragma unroll
            for (int j = 0; j < 4; ++j) gk[j] = fmaf(vp, wh.hk[b][j], gk[j]);
        }
        cf T[3];
        transfer_f32(wf, &gk[0], &gk[2], q.f.hi, sa, ca, amp * scale, T);
        const cf e = {cp, -sp};
#pragma unroll
        for (int c = 0; c < 3; ++c) h[c] = fadd(h[c], fmul(e, T[c]));
    }
    return any;
}


// delta = h/h0 - 1 of one walker at one edge record (the (2,2) mixed ratio of Sec. II B):
// rho = amp T h0inv (raw transfer, all frequency-only factors in h0inv), delta = (rho - 1) +
// rho (e^{-i dPhi} - 1) with dPhi in double-float; -1 outside the walker's support (h = 0)
__device__ __forceinline__ void edge_delta_mixed(const WalkerDF& wd, const WalkerF& wf, const MixEdge* pe, f2 tob,
                                                 cf dl[3])
{
    // the 80-byte record as five 128-bit loads
    const float4* p4 = reinterpret_cast<const float4*>(pe);
    const float4 r0 = p4[0], r1 = p4[1], r2 = p4[2], r3 = p4[3];
    MixEdge me;
    me.f = make_float2(r0.x, r0.y);
    me.f3 = make_float2(r0.z, r0.w);
    me.fm3 = make_float2(r1.x, r1.y);
    me.lnf3 = make_float2(r1.z, r1.w);
    me.phi0 = make_float2(r2.x, r2.y);
    me.h0inv[0] = make_float2(r2.z, r2.w);
    me.h0inv[1] = make_float2(r3.x, r3.y);
    me.h0inv[2] = make_float2(r3.z, r3.w);
    me.xs = p4[4];
    const FreqDF q = {ld_f2(me.f), ld_f2(me.f3), ld_f2(me.fm3), ld_f2(me.lnf3)};
    f2 Phi;
    float sa, ca, amp;
    if (phase_df<false, true>(wd, wf, q, tob, Phi, sa, ca, amp)) {
        float sh, ch;
        sincos_small(0.5f * reduce_phase(dd_add_lazy(Phi, {-me.phi0.x, -me.phi0.y})), &sh, &ch);
        const cf em1 = {-2.0f * sh * sh, -2.0f * sh * ch};   // e^{-i dPhi} - 1
        cf T[3];
        transfer_f32<true>(wf, wf.Ga, wf.Gb, me.xs.w, sa, ca, 1.0f, me.xs.x, me.xs.y, T, wf.Glo);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cf rho = fmul(fscale(T[c], amp), {me.h0inv[c].x, me.h0inv[c].y});
            dl[c] = fadd({rho.re - 1.0f, rho.im}, fmul(rho, em1));
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) dl[c] = {-1.0f, 0.0f};   // h = 0: r = 0
    }
}

// delta = h/h0 - 1 of one walker at edge e of a higher-mode reference, float32 ratio (Sec. II B
// with the template of Eq. 9 summed over the modes before the ratio): from the per-mode
// reference records (edge_mixed_hm_kernel), starting from the stored sum u - 1.  Modes with the
// same m share f2 = 2f/m, so the phase chain, t(f2), the orbit, the reference's phase and g: one
// chain and one transfer per distinct m, with the modes' factors summed weighted by v^{p_lm}
// (the transfer is linear in them) and the group's u summed in its first mode's record.
__device__ __forceinline__ void edge_delta_mixed_hm(const WalkerDF& wd, const WalkerF& wf, const WalkerHMF& wh,
                                                    const MixTables& mix, int e, uint32_t modes, f2 tob,
                                                    cf dl[3])
{
    const MixEdge me = mix.edge[e];
    const FreqDF q = {ld_f2(me.f), ld_f2(me.f3), ld_f2(me.fm3), ld_f2(me.lnf3)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 b = mix.hm_base[e * 3 + c];
        dl[c] = {b.x, b.y};
    }
    for (int grp = 0; grp < 4; ++grp) {
        const uint32_t gmask = modes & hm_group_mask(grp);
        if (!gmask) continue;
        const int b0 = __ffs(gmask) - 1;   // the group's first mode
        const MixModeHM mm = mix.hm[(int64_t)e * kHmModes + b0];
        const FreqDF q2 = mode_tables(q, b0);
        f2 Phi;
        float sa, ca, amp;
        if (phase_df<false, true>(wd, wf, q2, tob, Phi, sa, ca, amp)) {
            float sh, ch;
            sincos_small(0.5f * reduce_phase(dd_add_lazy(mode_phase(Phi, b0), {-mm.phi0.x, -mm.phi0.y})), &sh, &ch);
            const cf em1 = {-2.0f * sh * sh, -2.0f * sh * ch};   // e^{-i dPhi} - 1
            float gk[4] = {0.f, 0.f, 0.f, 0.f}, gl[4] = {0.f, 0.f, 0.f, 0.f};
            for (uint32_t bm = gmask; bm; bm &= bm - 1) {
                const int b = __ffs(bm) - 1;
                const float vp = mode_vpow(wd, q2, b);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    gk[j] = fmaf(vp, wh.hk[b][j], gk[j]);
                    gl[j] = fmaf(vp, wh.hklo[b][j], gl[j]);
                }
            }
            cf T[3];
            transfer_f32<true>(wf, &gk[0], &gk[2], me.xs.w, sa, ca, 1.0f, me.xs.x, me.xs.y, T, gl);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const cf u = {mm.u[c].x, mm.u[c].y};
                const cf ac = fsub(fmul(fscale(T[c], amp), {mm.g[c].x, mm.g[c].y}), u);
                dl[c] = fadd(dl[c], fadd(fadd(ac, fmul(ac, em1)), fmul(u, em1)));
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) dl[c] = fsub(dl[c], {mm.u[c].x, mm.u[c].y});
        }
    }
}

}  // namespace mbh


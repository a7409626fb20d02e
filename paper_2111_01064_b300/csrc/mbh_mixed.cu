// Mixed-precision path of libmbhlike (Katz, arXiv:2111.01064, Sec. II): the large phase
// Phi(f) = Psi(f) + 2 pi f k.c(t(f)) (up to ~1e7 rad) and t(f) are carried in double-float
// (float pairs, ~48 bits, mbh_df.cuh); amplitudes, the response, ratios and products are
// float32; sums are double-float or float64.
//
// B300 runs float64 FMA at 1/64 of the float32 rate, and its float64 pipe also carries
// conversions, compares and rounding; a float64 phase chain left this kernel bound by that
// pipe (84% busy, float32 pipe 12%).  The chain therefore runs on the float32 pipe:
//  - v = (pi M f)^{1/3} and ln v come from per-frequency tables (f^{1/3}, f^{-1/3}, ln f / 3)
//    times per-walker constants, so there is no cbrt/log per point;
//  - the orbital angle alpha(t) = alpha(t_ref) + dalpha with dalpha = 2 pi (t - t_ref)/yr:
//    sin/cos alpha(t_ref) are double-float per walker and the correction
//    (cos dalpha - 1, sin dalpha) is float32 from the half angle, accurate relative to its
//    own (small) size;
//  - the phase is reduced modulo 2 pi in double-float and only then rounded to float32.
// The heterodyne works in delta = r - 1 = (rho - 1) e^{-i dPhi} + (e^{-i dPhi} - 1), with
// rho = H/H0 the float32 ratio of the transfer parts and dPhi = Phi - Phi0 in double-float,
// and contracts the "1" part once in float64 (sum Re A0, sum B0).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "mbh_df.cuh"
#include "mbh_internal.cuh"
#include "mbh_model.cuh"
#include "mbh_pt.cuh"

using namespace mbh;

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

// Per-walker constants of the mixed path (Sec. II A parameter derivation), in float64: the
// large-phase constants (PN coefficients, the v and ln v scales, t_ref and the f_max
// references, the orbital angle at t_ref, the in-plane propagation components) are split
// into float pairs with integer operations (split_f64); the amplitude, polarisation and mode
// factors are rounded once to float32.  One thread per walker; the caller spreads walkers
// over full warps (a float64 warp instruction costs the same with 4 or 32 active lanes).
__device__ inline void walker_setup_mixed(const double* __restrict__ theta, int64_t W, int64_t i,
                                          WalkerDF& m, WalkerF& wf)
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
    m.c1 = split_f64(kTwoPi * tref - dpsi_max + (kxd * ca + kyd * sa), 0);   // with k.c(t_ref)
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

}  // namespace mbh

// ------------------------------------------------------------------------------------------
// self-test of the float32 device math
// ------------------------------------------------------------------------------------------
__global__ void selftest_math_kernel(int kind, const float* __restrict__ x, const float* __restrict__ y,
                                     int64_t n, float* __restrict__ o1, float* __restrict__ o2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (kind == 0) {
            float s, c;
            sincos_small(x[i], &s, &c);
            o1[i] = s;
            o2[i] = c;
        } else if (kind == 1) {
            o1[i] = sincf(x[i]);
        } else if (kind == 2) {
            o1[i] = sinc_diff(x[i], y[i]);
        } else if (kind == 3) {
            o1[i] = sinc_series<4>(x[i] * x[i]);
        } else {
            o1[i] = sinc_diff_series<4>(x[i], y[i]);
        }
    }
}

extern "C" mbh_status mbh_selftest_math(int32_t kind, const float* x_dev, const float* y_dev, int64_t n,
                                        float* o1_dev, float* o2_dev, void* stream)
{
    if (kind < 0 || kind > 4) return fail(MBH_EINVAL, "kind must be 0..4");
    if (n < 0) return fail(MBH_EINVAL, "n < 0");
    if (n == 0) return MBH_OK;
    if (!x_dev || !o1_dev || (kind == 0 && !o2_dev) || ((kind == 2 || kind == 4) && !y_dev))
        return fail(MBH_EINVAL, "NULL buffer");
    if (mbh_status s = check_device()) return s;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32);
    selftest_math_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(kind, x_dev, y_dev, n, o1_dev, o2_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "mbh_selftest_math");
}

// ------------------------------------------------------------------------------------------
// templates (complex64 storage)
// ------------------------------------------------------------------------------------------
constexpr int kTplThreadsM = 128;
constexpr int kTplPerThreadM = 4;

template <bool kHM>
__global__ void __launch_bounds__(kTplThreadsM)
    template_mixed_kernel(const double* __restrict__ theta, int64_t W, double f0, double df,
                          int64_t n, double t_obs, uint32_t modes, float2* __restrict__ h)
{
    __shared__ WalkerF wsf;
    __shared__ WalkerDF wsd;
    __shared__ WalkerHMF wsh;
    const f2 tob = split_d(t_obs);
    for (int64_t wi = blockIdx.y; wi < W; wi += gridDim.y) {
        __syncthreads();
        if (threadIdx.x == 0) {
            walker_setup_mixed(theta, W, wi, wsd, wsf);
            if (kHM) walker_setup_hm(theta, W, wi, wsh);
        }
        __syncthreads();
        const int64_t base = (int64_t)blockIdx.x * kTplThreadsM * kTplPerThreadM + threadIdx.x;
#pragma unroll
        for (int j = 0; j < kTplPerThreadM; ++j) {
            const int64_t k = base + (int64_t)j * kTplThreadsM;
            if (k < n) {
                const FreqDF q = freq_tables(f0 + (double)k * df);
                cf v[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                if (kHM)
                    point_mixed_hm(wsd, wsf, wsh, q, tob, 1.0f, modes, v);
                else
                    point_mixed(wsd, wsf, q, tob, 1.0f, v);
#pragma unroll
                for (int c = 0; c < 3; ++c) h[((int64_t)wi * 3 + c) * n + k] = make_float2(v[c].re, v[c].im);
            }
        }
    }
}

mbh_status mbh::launch_template_mixed(const mbh_grid* g, const double* theta, int64_t W, float2* h,
                                      cudaStream_t st, uint32_t modes)
{
    const int64_t per_block = (int64_t)kTplThreadsM * kTplPerThreadM;
    dim3 grid((unsigned)((g->n + per_block - 1) / per_block), (unsigned)std::min<int64_t>(W, 65535));
    if (modes == 1u)
        template_mixed_kernel<false><<<grid, kTplThreadsM, 0, st>>>(theta, W, g->f0, g->df, g->n, g->t_obs, modes, h);
    else
        template_mixed_kernel<true><<<grid, kTplThreadsM, 0, st>>>(theta, W, g->f0, g->df, g->n, g->t_obs, modes, h);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "template_mixed_kernel");
}

// ------------------------------------------------------------------------------------------
// direct likelihood, fused, mixed precision
// ------------------------------------------------------------------------------------------
constexpr int kDirThreadsM = 256;

// block (walker tile of T, frequency chunk).  The frequency tables and the float32 data of a
// grid point are loaded once and reused by the T walkers; each thread keeps its per-walker
// float64 sums in shared memory (a dynamically indexed register array would go to local
// memory), reduced per walker at the end.  Data and templates are in units where h/sigma is
// O(1) (float32 range); per-point products are float32, sums float64.
constexpr int kDirFlush = 16;   // points per float32 partial sum in the fused mixed pass

template <int T, bool kHM>
__global__ void __launch_bounds__(kDirThreadsM, 2)
    direct_fused_mixed_kernel(const double* __restrict__ theta, int64_t W, const float4* __restrict__ ft1,
                              const float4* __restrict__ ft2, const float4* __restrict__ ft3, double t_obs,
                              const float2* __restrict__ wd, const float* __restrict__ wv,
                              const float2* __restrict__ wdk, const float* __restrict__ wvk,
                              int64_t n, int64_t chunk, int nchunks, float inv_sigma, uint32_t modes,
                              double2* __restrict__ part)
{
    __shared__ WalkerDF wsd[T];
    __shared__ WalkerF wsf[T];
    __shared__ WalkerHMF wsh[kHM ? T : 1];
    __shared__ double2 acc[T][kDirThreadsM];
    __shared__ float2 facc[T][kDirThreadsM];
    __shared__ double sm[32 * 2];
    const int64_t w0 = (int64_t)blockIdx.x * T;
    const int ch = blockIdx.y;
    const int nt = (int)std::min<int64_t>(T, W - w0);
    if (threadIdx.x < nt) {
        walker_setup_mixed(theta, W, w0 + threadIdx.x, wsd[threadIdx.x], wsf[threadIdx.x]);
        if (kHM) walker_setup_hm(theta, W, w0 + threadIdx.x, wsh[threadIdx.x]);
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        acc[t][threadIdx.x] = make_double2(0.0, 0.0);
        facc[t][threadIdx.x] = make_float2(0.0f, 0.0f);
    }
    // t_obs split once into shared memory: a register copy that the compiler rematerialises
    // from the float64 parameter inside the point loop costs float64-pipe work at every point
    __shared__ f2 s_tob;
    if (threadIdx.x == 0) s_tob = split_d(t_obs);
    __syncthreads();
    const f2 tob = s_tob;
    const int64_t kb = (int64_t)ch * chunk, ke = std::min<int64_t>(n, kb + chunk);
    int since = 0;
    for (int64_t k = kb + threadIdx.x; k < ke; k += kDirThreadsM) {
        const float4 a = __ldg(ft1 + k), b = __ldg(ft2 + k);
        const FreqDF q = {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}, {b.z, b.w}};
        // (2,2): raw templates against the folded data (folded_data_kernel); higher modes: full
        // templates against the scaled data
        const float2* wdc = kHM ? wd : wdk;
        const float* wvc = kHM ? wv : wvk;
        float2 d[3];
        float v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            d[c] = __ldg(wdc + (int64_t)c * n + k);
            v[c] = __ldg(wvc + (int64_t)c * n + k);
        }
        const float4 xs = kHM ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(ft3 + k);
        for (int t = 0; t < nt; ++t) {
            cf h[3];
            const bool in = kHM ? point_mixed_hm(wsd[t], wsf[t], wsh[t], q, tob, inv_sigma, modes, h)
                                : point_mixed_raw(wsd[t], wsf[t], q, xs, tob, inv_sigma, h);
            if (in) {
                float pd = 0.0f, ph = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    pd += d[c].x * h[c].re + d[c].y * h[c].im;
                    ph += v[c] * (h[c].re * h[c].re + h[c].im * h[c].im);
                }
                float2 f = facc[t][threadIdx.x];
                f.x += pd;
                f.y += ph;
                facc[t][threadIdx.x] = f;
            }
        }
        // float32 partial sums of up to kDirFlush points go into the float64 accumulators (the
        // conversions and adds run on the float64 pipe: once per kDirFlush points, not per point)
        if (++since == kDirFlush) {
            since = 0;
            for (int t = 0; t < nt; ++t) {
                const float2 f = facc[t][threadIdx.x];
                double2 s2 = acc[t][threadIdx.x];
                s2.x += (double)f.x;
                s2.y += (double)f.y;
                acc[t][threadIdx.x] = s2;
                facc[t][threadIdx.x] = make_float2(0.0f, 0.0f);
            }
        }
    }
    for (int t = 0; t < nt; ++t) {
        const float2 f = facc[t][threadIdx.x];
        double2 s2 = acc[t][threadIdx.x];
        s2.x += (double)f.x;
        s2.y += (double)f.y;
        acc[t][threadIdx.x] = s2;
    }
    for (int t = 0; t < nt; ++t) {
        double r[2] = {acc[t][threadIdx.x].x, acc[t][threadIdx.x].y};
        block_sum<2>(r, sm);
        if (threadIdx.x == 0) {
            // the raw (2,2) templates used the float32 amp76: undo its rounding (a pure scale)
            const double fix = kHM ? 1.0 : 1.0 + (double)wsf[t].eps_amp76;
            part[(w0 + t) * nchunks + ch] = make_double2(r[0] * fix, r[1] * (fix * fix));
        }
    }
}

// frequency-only inputs of an edge, rounded once from float64: sin and cos of the one-link
// phase x = pi f L/c, and x
__device__ __forceinline__ float4 edge_xs(double f)
{
    const double x = kPi * kArmSec * f;
    double s, c;
    sincos(x, &s, &c);
    return make_float4((float)s, (float)c, 0.0f, (float)x);
}

__global__ void freq_table_kernel(double f0, double df, int64_t n, float4* __restrict__ t1,
                                  float4* __restrict__ t2, float4* __restrict__ t3)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double f = f0 + (double)k * df;
        const FreqDF q = freq_tables(f);
        t1[k] = make_float4(q.f.hi, q.f.lo, q.f3.hi, q.f3.lo);
        t2[k] = make_float4(q.fm3.hi, q.fm3.lo, q.lnf3.hi, q.lnf3.lo);
        t3[k] = edge_xs(f);
    }
}

// The fused mixed pass's data with the template's frequency-only factors folded in (float64,
// rounded once): with h_c = K_c H_c (H_c the raw float32 template of transfer_f32<true> and
// phase_df<.., true>, K_c as in the heterodyne's edge records, including f^{-7/6}),
// Re conj(D_c) h_c = Re conj(conj(K_c) D_c) H_c and |h_c|^2 V_c = |H_c|^2 |K_c|^2 V_c.
__global__ void folded_data_kernel(double f0, double df, int64_t n, double sigma, const double2* __restrict__ wd,
                                   const double* __restrict__ wv, float2* __restrict__ wdk,
                                   float* __restrict__ wvk)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double f = f0 + (double)k * df;
        const double x = kPi * kArmSec * f;
        double s1, c1, s3, c3;
        sincos(x, &s1, &c1);
        sincos(3.0 * x, &s3, &c3);
        const double wm = -2.0 * x * (2.0 * s1 * c1) * pow(f, -7.0 / 6.0);
        const double wr = wm * s3, wi = wm * c3;
        const double ar = 2.0 * s1 * s1, ai = 2.0 * s1 * c1;
        const double Kr[3] = {wr / kSqrt2, wr / kSqrt6, (wr * ar - wi * ai) / kSqrt3};
        const double Ki[3] = {wi / kSqrt2, wi / kSqrt6, (wr * ai + wi * ar) / kSqrt3};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 d = wd[c * n + k];
            const double dr = sigma * d.x, di = sigma * d.y;   // conj(K) D
            wdk[c * n + k] = make_float2((float)(Kr[c] * dr + Ki[c] * di), (float)(Kr[c] * di - Ki[c] * dr));
            wvk[c * n + k] = (float)(sigma * sigma * wv[c * n + k] * (Kr[c] * Kr[c] + Ki[c] * Ki[c]));
        }
    }
}

mbh_status mbh::make_freq_tables(mbh_data* D, cudaStream_t st)
{
    const int64_t n = D->grid.n;
    cudaError_t e = cudaMalloc(&D->ftab, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->ftab2, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->ftab3, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->wdk, sizeof(float2) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->wvk, sizeof(float) * 3 * n);
    if (e != cudaSuccess) return cuda_fail(e, "frequency tables");
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32);
    freq_table_kernel<<<blocks, 256, 0, st>>>(D->grid.f0, D->grid.df, n, D->ftab, D->ftab2, D->ftab3);
    folded_data_kernel<<<blocks, 256, 0, st>>>(D->grid.f0, D->grid.df, n, D->sigma, D->wd, D->wv, D->wdk, D->wvk);
    e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "frequency tables");
}

mbh_status mbh::launch_direct_fused_mixed(const mbh_data* data, const double* theta, int64_t W,
                                          double* out, cudaStream_t st, uint32_t modes)
{
    constexpr int T = 8;
    const int64_t tiles = (W + T - 1) / T;
    if (tiles > 0x7fffffff) return fail(MBH_EINVAL, "W too large");
    int64_t chunk;
    int nchunks;
    direct_chunks(data->grid.n, tiles, 1 << 14, chunk, nchunks);
    double2* part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, sizeof(double2) * W * nchunks, st);
    if (e != cudaSuccess) return cuda_fail(e, "direct_loglike_batch alloc");
    dim3 grid((unsigned)tiles, (unsigned)nchunks);
    if (modes == 1u)
        direct_fused_mixed_kernel<T, false><<<grid, kDirThreadsM, 0, st>>>(
            theta, W, data->ftab, data->ftab2, data->ftab3, data->grid.t_obs, data->wd32, data->wv32,
            data->wdk, data->wvk, data->grid.n, chunk, nchunks, (float)(1.0 / data->sigma), modes, part);
    else
        direct_fused_mixed_kernel<T, true><<<grid, kDirThreadsM, 0, st>>>(
            theta, W, data->ftab, data->ftab2, data->ftab3, data->grid.t_obs, data->wd32, data->wv32,
            data->wdk, data->wvk, data->grid.n, chunk, nchunks, (float)(1.0 / data->sigma), modes, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "direct_fused_mixed_kernel");
    return direct_finish(part, nchunks, W, data->dd, out, st);
}

// ------------------------------------------------------------------------------------------
// heterodyne reference tables
// ------------------------------------------------------------------------------------------
cudaError_t mbh::alloc_ref_tables(mbh_ref* R)
{
    const int E = R->E;
    cudaError_t e = cudaMalloc(&R->edges, sizeof(int64_t) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->fe, sizeof(double) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->invw, sizeof(double) * E);
    if (e == cudaSuccess) e = cudaMalloc(&R->summary, sizeof(double) * 18 * E);
    if (e == cudaSuccess) e = cudaMalloc(&R->h0e, sizeof(double2) * 3 * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->h0inv, sizeof(double2) * 3 * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->mix_edge, sizeof(MixEdge) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->mix_bin, sizeof(MixBin) * E);
    if (e == cudaSuccess) e = cudaMalloc(&R->mix_sums, sizeof(double) * 3);
    return e;
}

void mbh::free_ref_tables(mbh_ref* R)
{
    cudaFree(R->edges);
    cudaFree(R->fe);
    cudaFree(R->invw);
    cudaFree(R->summary);
    cudaFree(R->h0e);
    cudaFree(R->h0inv);
    cudaFree(R->mix_edge);
    cudaFree(R->mix_bin);
    cudaFree(R->mix_sums);
    if (R->mix_hm) cudaFree(R->mix_hm);
    if (R->mix_hm_base) cudaFree(R->mix_hm_base);
    free_x_tables(R);
}


// Edge records of the reference: its large phase Phi0 from the same double-float chain and edge
// tables as the walkers (so that Phi - Phi0 cancels exactly for the reference itself), and
// 1/H0 with H0 = h0 e^{+i Phi0}, h0 the float64 reference template at the edge: the walkers'
// ratio r = H e^{-i(Phi - Phi0)}/H0 is then h/h0 with the exact h0.  (An H0 from the walkers'
// own float32 chain would put its rounding into the ratio of every walker alike: a bias of
// ~1e-7 of <h|h> shared by the whole batch.)
__global__ void edge_mixed_kernel(const double* __restrict__ theta0, double t_obs,
                                  const double* __restrict__ fe, int n_edges,
                                  const double2* __restrict__ h0e, MixEdge* __restrict__ out,
                                  double* __restrict__ eps0)
{
    __shared__ WalkerDF wd;
    __shared__ WalkerF wf;
    if (threadIdx.x == 0) {
        walker_setup_mixed(theta0, 1, 0, wd, wf);
        *eps0 = 0.0;   // h0 is exact: no float32 amplitude on the reference side
    }
    __syncthreads();
    const f2 tob = split_d(t_obs);
    for (int e = threadIdx.x; e < n_edges; e += blockDim.x) {
        const FreqDF q = freq_tables(fe[e]);
        MixEdge m;
        m.f = make_float2(q.f.hi, q.f.lo);
        m.f3 = make_float2(q.f3.hi, q.f3.lo);
        m.fm3 = make_float2(q.fm3.hi, q.fm3.lo);
        m.lnf3 = make_float2(q.lnf3.hi, q.lnf3.lo);
        m.xs = edge_xs(fe[e]);
        f2 Phi = {0.0f, 0.0f};
        float sa, ca, amp;
        phase_df<true, true>(wd, wf, q, tob, Phi, sa, ca, amp);   // defined at every edge
        m.phi0 = make_float2(Phi.hi, Phi.lo);
        double sp, cp;
        sincos((double)Phi.hi + (double)Phi.lo, &sp, &cp);
        // frequency-only factors of the template (transfer_f32<true> and phase_df<.., true>):
        // W = (1 - D^2)(-x) e^{-ix} = -2 x sin 2x (sin 3x, cos 3x), 1 - D = 2 sin x (sin x, cos x),
        // K_A = W/sqrt2, K_E = W/sqrt6, K_T = W (1 - D)/sqrt3, all times f^{-7/6}
        const double x = kPi * kArmSec * fe[e];
        double s1, c1, s3, c3;
        sincos(x, &s1, &c1);
        sincos(3.0 * x, &s3, &c3);
        const double wm = -2.0 * x * (2.0 * s1 * c1) * pow(fe[e], -7.0 / 6.0);
        const double wr = wm * s3, wi = wm * c3;
        const double ar = 2.0 * s1 * s1, ai = 2.0 * s1 * c1;
        const double2 K[3] = {make_double2(wr / kSqrt2, wi / kSqrt2), make_double2(wr / kSqrt6, wi / kSqrt6),
                              make_double2((wr * ar - wi * ai) / kSqrt3, (wr * ai + wi * ar) / kSqrt3)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // 1/H0 in float64: |H0| is ~1e-20..1e-30 in strain units, so |H0|^2 underflows
            // float32, while 1/H0 itself (~1e20..1e30) is a normal float32
            // times the factors the walkers' raw transfer and amplitude leave out (K below)
            const double2 h = h0e[e * 3 + c];
            const double hr = h.x * cp - h.y * sp, hi = h.x * sp + h.y * cp;
            const double m2 = hr * hr + hi * hi;
            const double ir = hr / m2, ii = -hi / m2;
            m.h0inv[c] = m2 > 0.0 ? make_float2((float)(K[c].x * ir - K[c].y * ii), (float)(K[c].x * ii + K[c].y * ir))
                                  : make_float2(0.f, 0.f);
        }
        out[e] = m;
    }
}

// Higher-mode reference: per edge and mode the mode's large phase Phi0_lm from the walkers'
// double-float chain (defined also outside the mode's support), and per channel
// u = h0_lm/h0 and g = K f2^{-7/6} e^{-i Phi0_lm}/h0 in float64 from the exact float64 mode
// templates h0_lm (h0 = their sum), K the frequency-only factors of the walkers' raw transfer
// and f2 = 2f/m (whose f2^{-7/6} the walkers' amplitude leaves out); base = sum u - 1 of the
// float32 u (float64 sum, rounded once: the float32 u do not sum to 1 exactly, and the offset
// would be shared by every walker), -1 where h0 = 0 (r = 0 there).  A walker's delta = r - 1
// is then
//   base + sum_lm [a + a (e^{-i dPhi_lm} - 1) + u (e^{-i dPhi_lm} - 1)],  a = H_lm g - u,
// with H_lm its raw float32 mode template; a mode outside the walker's support contributes -u.
__global__ void edge_mixed_hm_kernel(const double* __restrict__ theta0, double t_obs, uint32_t modes,
                                     const double* __restrict__ fe, int n_edges, MixEdge* __restrict__ out,
                                     MixModeHM* __restrict__ hm, float2* __restrict__ base,
                                     double* __restrict__ eps0)
{
    __shared__ WalkerDF wd;
    __shared__ WalkerF wf;
    __shared__ Walker w64;
    if (threadIdx.x == 0) {
        walker_setup_mixed(theta0, 1, 0, wd, wf);
        walker_setup(theta0, 1, 0, w64, modes);
        *eps0 = 0.0;   // h0 is exact: no float32 amplitude on the reference side
    }
    __syncthreads();
    const f2 tob = split_d(t_obs);
    for (int e = threadIdx.x; e < n_edges; e += blockDim.x) {
        const double f = fe[e];
        const FreqDF q = freq_tables(f);
        MixEdge me{};
        me.f = make_float2(q.f.hi, q.f.lo);
        me.f3 = make_float2(q.f3.hi, q.f3.lo);
        me.fm3 = make_float2(q.fm3.hi, q.fm3.lo);
        me.lnf3 = make_float2(q.lnf3.hi, q.lnf3.lo);
        me.xs = edge_xs(f);
        out[e] = me;
        // frequency-only factors (as the (2,2) records, without f^{-7/6}, which goes per mode)
        const double x = kPi * kArmSec * f;
        double s1, c1, s3, c3;
        sincos(x, &s1, &c1);
        sincos(3.0 * x, &s3, &c3);
        const double wm = -2.0 * x * (2.0 * s1 * c1);
        const double wr = wm * s3, wi = wm * c3;
        const double ar = 2.0 * s1 * s1, ai = 2.0 * s1 * c1;
        const double Kr[3] = {wr / kSqrt2, wr / kSqrt6, (wr * ar - wi * ai) / kSqrt3};
        const double Ki[3] = {wi / kSqrt2, wi / kSqrt6, (wr * ai + wi * ar) / kSqrt3};
        cd h0m[kHmModes][3], h0[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        double gr[kHmModes], gi[kHmModes];   // f2^{-7/6} e^{-i Phi0_lm}
        for (int b = 0; b < kHmModes; ++b) {
            for (int c = 0; c < 3; ++c) h0m[b][c] = {0.0, 0.0};
            gr[b] = gi[b] = 0.0;
            MixModeHM mm{};
            if (modes & (1u << b)) {
                if (mode_point_f64(w64, b, f, t_obs, h0m[b]))
                    for (int c = 0; c < 3; ++c) h0[c] = cadd(h0[c], h0m[b][c]);
                const FreqDF q2 = mode_tables(q, b);
                f2 Phi;
                float sa, ca, amp;
                phase_df<true, true>(wd, wf, q2, tob, Phi, sa, ca, amp);
                const f2 P = mode_phase(Phi, b);
                mm.phi0 = make_float2(P.hi, P.lo);
                double sp, cp;
                sincos((double)P.hi + (double)P.lo, &sp, &cp);
                const double a = pow(2.0 * f / hm_m(b), -7.0 / 6.0);
                gr[b] = a * cp;
                gi[b] = -a * sp;
            }
            hm[(int64_t)e * kHmModes + b] = mm;
        }
        for (int c = 0; c < 3; ++c) {
            const double m2 = h0[c].re * h0[c].re + h0[c].im * h0[c].im;
            base[e * 3 + c] = make_float2(-1.0f, 0.0f);
            if (!(m2 > 0.0)) continue;
            double sur = -1.0, sui = 0.0;   // sum of the stored u, minus 1
            const double ir = h0[c].re / m2, ii = -h0[c].im / m2;   // 1/h0
            // per group of modes with the same m (same phase and g), the u summed into the
            // record of its first mode, which the kernel reads for the whole group
            for (int grp = 0; grp < 4; ++grp) {
                const uint32_t gmask = modes & hm_group_mask(grp);
                if (!gmask) continue;
                const int b0 = __ffs(gmask) - 1;
                double usr = 0.0, usi = 0.0;
                for (uint32_t bm = gmask; bm; bm &= bm - 1) {
                    const cd hb = h0m[__ffs(bm) - 1][c];
                    usr += hb.re * ir - hb.im * ii;
                    usi += hb.re * ii + hb.im * ir;
                }
                MixModeHM& mm = hm[(int64_t)e * kHmModes + b0];
                mm.u[c] = make_float2((float)usr, (float)usi);
                sur += (double)mm.u[c].x;
                sui += (double)mm.u[c].y;
                // K e'/h0, e' = f2^{-7/6} e^{-i Phi0_lm}
                const double er = Kr[c] * gr[b0] - Ki[c] * gi[b0], ei = Kr[c] * gi[b0] + Ki[c] * gr[b0];
                mm.g[c] = make_float2((float)(er * ir - ei * ii), (float)(er * ii + ei * ir));
            }
            base[e * 3 + c] = make_float2((float)sur, (float)sui);
        }
    }
}

// Bin records: the summary data of each channel with the contraction's constant factors folded
// in (float64, rounded once): from (A0, A1, B0, B1) as (q0, q1, q2, q3, q4, q5) and w = f_hi - f_lo,
// (q0/2, q1/2, q2/w, q3/w, q4/4, q5/w) for contract_bin.
__global__ void bin_mixed_kernel(const double* __restrict__ summary, const double* __restrict__ invw,
                                 int E, MixBin* __restrict__ out, double* __restrict__ sums)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < E) {
        MixBin m;
        const double iw = invw[b];
        const double fold[6] = {0.5, 0.5, iw, iw, 0.25, iw};
#pragma unroll
        for (int j = 0; j < 18; ++j) m.q[j] = (float)(summary[(int64_t)b * 18 + j] * fold[j % 6]);
        m.pad[0] = m.pad[1] = 0.0f;
        out[b] = m;
    }
    if (b == 0) {
        double a = 0.0, bb = 0.0;
        for (int i = 0; i < E; ++i)
            for (int c = 0; c < 3; ++c) {
                a += summary[(int64_t)i * 18 + 6 * c + 0];
                bb += summary[(int64_t)i * 18 + 6 * c + 4];
            }
        sums[0] = a;
        sums[1] = bb;
    }
}

cudaError_t mbh::prepare_mixed_tables(mbh_ref* R, cudaStream_t st)
{
    const int E = R->E;
    if (R->modes == 1u) {
        edge_mixed_kernel<<<1, 256, 0, st>>>(R->theta0_dev, R->grid.t_obs, R->fe, E + 1, R->h0e,
                                             R->mix_edge, R->mix_sums + 2);
    } else {
        cudaError_t e = cudaMalloc(&R->mix_hm, sizeof(MixModeHM) * kHmModes * (E + 1));
        if (e == cudaSuccess) e = cudaMalloc(&R->mix_hm_base, sizeof(float2) * 3 * (E + 1));
        if (e != cudaSuccess) return e;
        edge_mixed_hm_kernel<<<1, 128, 0, st>>>(R->theta0_dev, R->grid.t_obs, R->modes, R->fe, E + 1,
                                                R->mix_edge, R->mix_hm, R->mix_hm_base, R->mix_sums + 2);
    }
    bin_mixed_kernel<<<(E + 127) / 128, 128, 0, st>>>(R->summary, R->invw, E, R->mix_bin, R->mix_sums);
    cudaError_t e = cudaGetLastError();
    double sums[3];
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums, R->mix_sums, sizeof sums, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        R->mix.edge = R->mix_edge;
        R->mix.bin = R->mix_bin;
        R->mix.sumA0 = sums[0];
        R->mix.sumB0 = sums[1];
        R->mix.hm = R->mix_hm;
        R->mix.hm_base = R->mix_hm_base;
        R->mix.amp_eps0 = sums[2];
    }
    return e;
}

// Contribution of one bin to <d|h> and <h|h> (Eqs. 14, 17, without the 4 and the "1" parts), from delta at
// its low (dp) and high (dl) edge: with d0 = (dp + dl)/2, d1 = (dl - dp)/w per channel,
//   <d|h>: q0 d0r + q1 d0i + q2 d1r + q3 d1i,
//   <h|h>: q4 (2 d0r + |d0|^2) + 2 q5 (d1r + Re(d0 conj(d1)))   [first order, Eq. 17 as printed]
// evaluated in s = dp + dl, t = dl - dp with the record's folded factors (bin_mixed_kernel).
__device__ __forceinline__ void contract_bin(const MixBin& mb, const cf dp[3], const cf dl[3], float& bd,
                                             float& bh)
{
    // the record as five 128-bit loads (18 weights and 2 pad floats)
    float qa[20];
    const float4* q4 = reinterpret_cast<const float4*>(&mb);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float4 t = q4[k];
        qa[4 * k] = t.x;
        qa[4 * k + 1] = t.y;
        qa[4 * k + 2] = t.z;
        qa[4 * k + 3] = t.w;
    }
    bd = 0.0f;
    bh = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float sr = dp[c].re + dl[c].re, si = dp[c].im + dl[c].im;
        const float tr = dl[c].re - dp[c].re, ti = dl[c].im - dp[c].im;
        const float* q = qa + 6 * c;
        bd = fmaf(q[0], sr, fmaf(q[1], si, fmaf(q[2], tr, fmaf(q[3], ti, bd))));
        bh = fmaf(q[4], fmaf(si, si, sr * (4.0f + sr)), fmaf(q[5], fmaf(si, ti, tr * (2.0f + sr)), bh));
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

// A walker's <d|h>, <h|h> partial sums (float pairs) with the tail edge E, when the edge loop
// left it out: evaluated here, its bin E - 1 contracted against the carried delta at E - 1 and
// added last (the same order for every block size and launch mode)
__device__ __forceinline__ float4 tail_sums(const SrcDesc& S, const WalkerDF& wd, const WalkerF& wf, f2 tob,
                                            const cf dprev[3], bool tail, float4 v)
{
    if (!tail) return v;
    const int E = S.E;
    cf dl[3], dp[3];
    edge_delta_mixed(wd, wf, S.mix.edge + E, tob, dl);
#pragma unroll
    for (int c = 0; c < 3; ++c) dp[c] = dprev[c];
    float bd, bh;
    contract_bin(S.mix.bin[E - 1], dp, dl, bd, bh);
    f2 adh = {v.x, v.y}, ahh = {v.z, v.w};
    df_acc(adh, {bd, 0.0f});
    df_acc(ahh, {bh, 0.0f});
    return make_float4(adh.hi, adh.lo, ahh.hi, ahh.lo);
}

// ------------------------------------------------------------------------------------------
// heterodyne likelihood, mixed precision
// ------------------------------------------------------------------------------------------
// Each heterodyne kernel comes in two register budgets: het_*_kernel (power-of-two blocks)
// leaves the register count to the compiler (~96-118), het_*_kernel_capped (blocks of 96,
// 160, 224) is compiled for about 28 resident warps per SM (72 registers, a few bytes spilled):
// at 8 threads per walker 16384 walkers then fit in one wave (586 blocks of 224 threads on
// 148 x 4 slots) instead of the 1.4 waves that 96 registers allow.
template <int G, int BLOCK>
__device__ __forceinline__ void het_mixed_body(const HetLaunch& L)
{
    constexpr int WPB = BLOCK / G;
    __shared__ WalkerDF wsd[WPB];
    __shared__ WalkerF wsf[WPB];
    __shared__ float4 sums[WPB];   // per walker <d|h>, <h|h> partial sums (float pairs)
    __shared__ cf tailc[WPB][3];   // per walker delta at edge E - 1, for the tail edge
    const int lw = threadIdx.x / G, lane = threadIdx.x % G;
    for (int tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
        int s = 0;
        while (s + 1 < L.n_src && L.src[s + 1].tile_begin <= tile) ++s;
        const SrcDesc& S = L.src[s];
        const int64_t w0 = S.w_begin + (int64_t)(tile - S.tile_begin) * WPB;
        const int64_t wi = w0 + lw;
        const bool active = wi < S.w_end;
        __syncthreads();
        // setup with consecutive threads (full warps): a float64 warp instruction costs the
        // same whether 4 or 32 of its lanes are active
        for (int j = threadIdx.x; j < WPB; j += BLOCK)
            if (w0 + j < S.w_end) walker_setup_mixed(L.theta, L.W, w0 + j, wsd[j], wsf[j]);
        __syncthreads();
        const int E = S.E;
        const f2 tob = {S.tob_hi, S.tob_lo};
        f2 adh = {0.0f, 0.0f}, ahh = {0.0f, 0.0f};
        cf carry[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        // (E + 1) % G == 1 leaves one edge per walker for a last round with one active lane per
        // walker: that edge goes to the block-wide tail in the epilogue (consecutive threads)
        const bool tail = G > 1 && E >= 1 && (E + 1) % G == 1;
        const int rounds = tail ? E / G : (E + 1 + G - 1) / G;
        for (int r = 0; r < rounds; ++r) {
            const int e = r * G + lane;
            cf dl[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            const bool ok = active && e <= E && MBH_IN_RANGE(L.status, e, (long long)S.E_check + 1, kKernHetF32, s);
            if (ok) edge_delta_mixed(wsd[lw], wsf[lw], S.mix.edge + e, tob, dl);
            cf dp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dp[c].re = __shfl_up_sync(0xffffffffu, dl[c].re, 1, G);
                dp[c].im = __shfl_up_sync(0xffffffffu, dl[c].im, 1, G);
                if (lane == 0) dp[c] = carry[c];
                carry[c].re = __shfl_sync(0xffffffffu, dl[c].re, G - 1, G);
                carry[c].im = __shfl_sync(0xffffffffu, dl[c].im, G - 1, G);
            }
            if (ok && e >= 1) {
                float bd, bh;
                contract_bin(S.mix.bin[e - 1], dp, dl, bd, bh);
                df_acc(adh, {bd, 0.0f});
                df_acc(ahh, {bh, 0.0f});
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const f2 odh = {__shfl_down_sync(0xffffffffu, adh.hi, o, G), __shfl_down_sync(0xffffffffu, adh.lo, o, G)};
            const f2 ohh = {__shfl_down_sync(0xffffffffu, ahh.hi, o, G), __shfl_down_sync(0xffffffffu, ahh.lo, o, G)};
            df_acc(adh, odh);
            df_acc(ahh, ohh);
        }
        // float64 epilogue on consecutive threads (as the setup: a float64 warp instruction costs
        // the same for 32/G or 32 walkers)
        if (lane == 0) {
            sums[lw] = make_float4(adh.hi, adh.lo, ahh.hi, ahh.lo);
#pragma unroll
            for (int c = 0; c < 3; ++c) tailc[lw][c] = carry[c];   // delta at edge E - 1 (tail)
        }
        __syncthreads();
        for (int j = threadIdx.x; j < WPB; j += BLOCK)
            if (w0 + j < S.w_end) {
                const float4 v = tail_sums(S, wsd[j], wsf[j], tob, tailc[j], tail, sums[j]);
                const double fix = amp_fix(wsf[j].eps_amp76, S.mix.amp_eps0);
                const double dh = 4.0 * (S.mix.sumA0 + df_to_double({v.x, v.y})) * fix;
                const double hh = 4.0 * (S.mix.sumB0 + df_to_double({v.z, v.w})) * (fix * fix);
                L.out[w0 + j] = -0.5 * (S.dd + hh - 2.0 * dh);
                L.out[L.W + w0 + j] = dh;
                L.out[2 * L.W + w0 + j] = hh;
            }
    }
}


template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK) het_mixed_kernel(const __grid_constant__ HetLaunch L)
{
    het_mixed_body<G, BLOCK>(L);
}

template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 896 / BLOCK) het_mixed_kernel_capped(const __grid_constant__ HetLaunch L)
{
    het_mixed_body<G, BLOCK>(L);
}

// Higher-mode heterodyne (Sec. II B with the template of Eq. 9 summed over modes before the
// ratio), mixed precision; layout and reductions as het_mixed_kernel, delta from the
// per-mode reference tables (edge_mixed_hm_kernel).  The register cap (640 threads per SM,
// 102 registers) fits five 128-thread blocks per SM against four uncapped, without spills.
template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 640 / BLOCK)
    het_mixed_hm_kernel(const __grid_constant__ HetLaunch L)
{
    constexpr int WPB = BLOCK / G;
    __shared__ WalkerDF wsd[WPB];
    __shared__ WalkerF wsf[WPB];
    __shared__ WalkerHMF wsh[WPB];
    __shared__ float4 sums[WPB];   // per walker <d|h>, <h|h> partial sums (float pairs)
    const int lw = threadIdx.x / G, lane = threadIdx.x % G;
    for (int tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
        int s = 0;
        while (s + 1 < L.n_src && L.src[s + 1].tile_begin <= tile) ++s;
        const SrcDesc& S = L.src[s];
        const int64_t w0 = S.w_begin + (int64_t)(tile - S.tile_begin) * WPB;
        const int64_t wi = w0 + lw;
        const bool active = wi < S.w_end;
        __syncthreads();
        for (int j = threadIdx.x; j < WPB; j += BLOCK)
            if (w0 + j < S.w_end) {
                walker_setup_mixed(L.theta, L.W, w0 + j, wsd[j], wsf[j]);
                walker_setup_hm(L.theta, L.W, w0 + j, wsh[j]);
            }
        __syncthreads();
        const int E = S.E;
        const uint32_t modes = S.modes;
        const f2 tob = {S.tob_hi, S.tob_lo};
        f2 adh = {0.0f, 0.0f}, ahh = {0.0f, 0.0f};
        cf carry[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        const int rounds = (E + 1 + G - 1) / G;
        for (int r = 0; r < rounds; ++r) {
            const int e = r * G + lane;
            cf dl[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            if (active && e <= E) {
                const MixEdge me = S.mix.edge[e];
                const FreqDF q = {ld_f2(me.f), ld_f2(me.f3), ld_f2(me.fm3), ld_f2(me.lnf3)};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 b = S.mix.hm_base[e * 3 + c];
                    dl[c] = {b.x, b.y};
                }
                // Modes with the same m share f2 = 2f/m, so the phase chain, t(f2), the orbit, the
                // reference's phase and g: one chain and one transfer per distinct m, with the
                // modes' factors summed weighted by v^{p_lm} (the transfer is linear in them) and
                // the group's u summed in its first mode's record (edge_mixed_hm_kernel).
                for (int grp = 0; grp < 4; ++grp) {
                    const uint32_t gmask = modes & hm_group_mask(grp);
                    if (!gmask) continue;
                    const int b0 = __ffs(gmask) - 1;   // the group's first mode
                    const MixModeHM mm = S.mix.hm[(int64_t)e * kHmModes + b0];
                    const FreqDF q2 = mode_tables(q, b0);
                    f2 Phi;
                    float sa, ca, amp;
                    if (phase_df<false, true>(wsd[lw], wsf[lw], q2, tob, Phi, sa, ca, amp)) {
                        float sh, ch;
                        sincos_small(0.5f * reduce_phase(dd_add_lazy(mode_phase(Phi, b0), {-mm.phi0.x, -mm.phi0.y})),
                                     &sh, &ch);
                        const cf em1 = {-2.0f * sh * sh, -2.0f * sh * ch};   // e^{-i dPhi} - 1
                        float gk[4] = {0.f, 0.f, 0.f, 0.f}, gl[4] = {0.f, 0.f, 0.f, 0.f};
                        for (uint32_t bm = gmask; bm; bm &= bm - 1) {
                            const int b = __ffs(bm) - 1;
                            const float vp = mode_vpow(wsd[lw], q2, b);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                gk[j] = fmaf(vp, wsh[lw].hk[b][j], gk[j]);
                                gl[j] = fmaf(vp, wsh[lw].hklo[b][j], gl[j]);
                            }
                        }
                        cf T[3];
                        transfer_f32<true>(wsf[lw], &gk[0], &gk[2], me.xs.w, sa, ca, 1.0f, me.xs.x, me.xs.y, T, gl);
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
            cf dp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dp[c].re = __shfl_up_sync(0xffffffffu, dl[c].re, 1, G);
                dp[c].im = __shfl_up_sync(0xffffffffu, dl[c].im, 1, G);
                if (lane == 0) dp[c] = carry[c];
                carry[c].re = __shfl_sync(0xffffffffu, dl[c].re, G - 1, G);
                carry[c].im = __shfl_sync(0xffffffffu, dl[c].im, G - 1, G);
            }
            if (active && e >= 1 && e <= E) {
                float bd, bh;
                contract_bin(S.mix.bin[e - 1], dp, dl, bd, bh);
                df_acc(adh, {bd, 0.0f});
                df_acc(ahh, {bh, 0.0f});
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const f2 odh = {__shfl_down_sync(0xffffffffu, adh.hi, o, G), __shfl_down_sync(0xffffffffu, adh.lo, o, G)};
            const f2 ohh = {__shfl_down_sync(0xffffffffu, ahh.hi, o, G), __shfl_down_sync(0xffffffffu, ahh.lo, o, G)};
            df_acc(adh, odh);
            df_acc(ahh, ohh);
        }
        // float64 epilogue on consecutive threads (as the setup: a float64 warp instruction costs
        // the same for 32/G or 32 walkers)
        if (lane == 0) sums[lw] = make_float4(adh.hi, adh.lo, ahh.hi, ahh.lo);
        __syncthreads();
        for (int j = threadIdx.x; j < WPB; j += BLOCK)
            if (w0 + j < S.w_end) {
                const float4 v = sums[j];
                const double fix = amp_fix(wsf[j].eps_amp76, S.mix.amp_eps0);
                const double dh = 4.0 * (S.mix.sumA0 + df_to_double({v.x, v.y})) * fix;
                const double hh = 4.0 * (S.mix.sumB0 + df_to_double({v.z, v.w})) * (fix * fix);
                L.out[w0 + j] = -0.5 * (S.dd + hh - 2.0 * dh);
                L.out[L.W + w0 + j] = dh;
                L.out[2 * L.W + w0 + j] = hh;
            }
    }
}


// Sampler half step fused with the heterodyne likelihood (the sampler of Sec. III driving the
// likelihood of Sec. II B): the walker setup builds moving walker w's proposal from the
// ensemble state (pt::propose_item) and sets the walker up from theta(Y); the edge loop is
// het_mixed_kernel's; the epilogue applies the tempered acceptance (pt::accept_test) and
// updates the state and counters.  Walker index w = the half step's item t W/2 + k'.
template <int G, int BLOCK>
__device__ __forceinline__ void het_mixed_pt_body(const HetLaunch& L)
{
    constexpr int WPB = BLOCK / G;
    __shared__ WalkerDF wsd[WPB];
    __shared__ WalkerF wsf[WPB];
    __shared__ double ys[WPB][pt::kPar];
    __shared__ double facs[WPB];
    __shared__ int32_t flags[WPB];
    __shared__ float4 sums[WPB];   // per walker <d|h>, <h|h> partial sums (float pairs)
    __shared__ cf tailc[WPB][3];   // per walker delta at edge E - 1, for the tail edge
    const pt::PtArgs& A = *static_cast<const pt::PtArgs*>(L.pt);
    const int half = L.pt_half;
    const int lw = threadIdx.x / G, lane = threadIdx.x % G;
    for (int tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
        int s = 0;   // ensemble of this tile
        while (s + 1 < L.n_src && L.src[s + 1].tile_begin <= tile) ++s;
        const SrcDesc& S = L.src[s];
        const int64_t w0 = S.w_begin + (int64_t)(tile - S.tile_begin) * WPB;
        const int64_t wi = w0 + lw;
        const bool active = wi < S.w_end;
        __syncthreads();
        for (int j = threadIdx.x; j < WPB; j += BLOCK)
            if (w0 + j < S.w_end) {
                double v[pt::kPar], th[pt::kPar], fac;
                int32_t flag;
                pt::propose_item(A, half, (int32_t)(w0 + j), *A.step, v, th, fac, flag);
#pragma unroll
                for (int p = 0; p < pt::kPar; ++p) ys[j][p] = v[p];
                facs[j] = fac;
                flags[j] = flag;
                walker_setup_mixed(th, 1, 0, wsd[j], wsf[j]);
            }
        __syncthreads();
        const int E = S.E;
        const f2 tob = {S.tob_hi, S.tob_lo};
        f2 adh = {0.0f, 0.0f}, ahh = {0.0f, 0.0f};
        cf carry[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        // (E + 1) % G == 1 leaves one edge per walker for a last round with one active lane per
        // walker: that edge goes to the block-wide tail in the epilogue (consecutive threads)
        const bool tail = G > 1 && E >= 1 && (E + 1) % G == 1;
        const int rounds = tail ? E / G : (E + 1 + G - 1) / G;
        for (int r = 0; r < rounds; ++r) {
            const int e = r * G + lane;
            cf dl[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            const bool ok = active && e <= E && MBH_IN_RANGE(L.status, e, (long long)S.E_check + 1, kKernHetF32, s);
            if (ok) edge_delta_mixed(wsd[lw], wsf[lw], S.mix.edge + e, tob, dl);
            cf dp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dp[c].re = __shfl_up_sync(0xffffffffu, dl[c].re, 1, G);
                dp[c].im = __shfl_up_sync(0xffffffffu, dl[c].im, 1, G);
                if (lane == 0) dp[c] = carry[c];
                carry[c].re = __shfl_sync(0xffffffffu, dl[c].re, G - 1, G);
                carry[c].im = __shfl_sync(0xffffffffu, dl[c].im, G - 1, G);
            }
            if (ok && e >= 1) {
                float bd, bh;
                contract_bin(S.mix.bin[e - 1], dp, dl, bd, bh);
                df_acc(adh, {bd, 0.0f});
                df_acc(ahh, {bh, 0.0f});
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const f2 odh = {__shfl_down_sync(0xffffffffu, adh.hi, o, G), __shfl_down_sync(0xffffffffu, adh.lo, o, G)};
            const f2 ohh = {__shfl_down_sync(0xffffffffu, ahh.hi, o, G), __shfl_down_sync(0xffffffffu, ahh.lo, o, G)};
            df_acc(adh, odh);
            df_acc(ahh, ohh);
        }
        // float64 epilogue and acceptance on consecutive threads (full warps)
        if (lane == 0) {
            sums[lw] = make_float4(adh.hi, adh.lo, ahh.hi, ahh.lo);
#pragma unroll
            for (int c = 0; c < 3; ++c) tailc[lw][c] = carry[c];   // delta at edge E - 1 (tail)
        }
        __syncthreads();
        for (int j = threadIdx.x; j < WPB; j += BLOCK)
            if (w0 + j < S.w_end) {
                const float4 v = tail_sums(S, wsd[j], wsf[j], tob, tailc[j], tail, sums[j]);
                const double fix = amp_fix(wsf[j].eps_amp76, S.mix.amp_eps0);
                const double dh = 4.0 * (S.mix.sumA0 + df_to_double({v.x, v.y})) * fix;
                const double hh = 4.0 * (S.mix.sumB0 + df_to_double({v.z, v.w})) * (fix * fix);
                const double lnl = -0.5 * (S.dd + hh - 2.0 * dh);
                int32_t col;
                int t, cb;
                const int32_t flag = flags[j];
                const int kind = flag >> 1;
                const bool acc = pt::accept_test(A, half, (int32_t)(w0 + j), lnl, facs[j], flag, col, t, cb);
                atomicAdd(&A.counters[cb + t * 4 + kind], 1ull);
                if (acc) {
                    atomicAdd(&A.counters[cb + 4 * A.T + t * 4 + kind], 1ull);
                    const int64_t N = (int64_t)A.n_ens * A.T * A.W;
#pragma unroll
                    for (int p = 0; p < pt::kPar; ++p) A.x[p * N + col] = ys[j][p];
                    A.out[col] = lnl;
                    A.out[N + col] = dh;
                    A.out[2 * N + col] = hh;
                }
            }
    }
}

template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK) het_mixed_pt_kernel(const __grid_constant__ HetLaunch L)
{
    het_mixed_pt_body<G, BLOCK>(L);
}

template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 896 / BLOCK) het_mixed_pt_kernel_capped(const __grid_constant__ HetLaunch L)
{
    het_mixed_pt_body<G, BLOCK>(L);
}

namespace {
template <int G, int BLOCK>
cudaError_t launch_het_mixed(const HetLaunch& L, int grid, cudaStream_t st)
{
    if constexpr (BLOCK % 64 == 0)
        het_mixed_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    else
        het_mixed_kernel_capped<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}

template <int G, int BLOCK>
const void* het_mixed_fn()
{
    if constexpr (BLOCK % 64 == 0)
        return (const void*)&het_mixed_kernel<G, BLOCK>;
    else
        return (const void*)&het_mixed_kernel_capped<G, BLOCK>;
}

template <int G, int BLOCK>
const void* het_mixed_pt_fn()
{
    if constexpr (BLOCK % 64 == 0)
        return (const void*)&het_mixed_pt_kernel<G, BLOCK>;
    else
        return (const void*)&het_mixed_pt_kernel_capped<G, BLOCK>;
}

template <int G, int BLOCK>
cudaError_t launch_het_mixed_hm(const HetLaunch& L, int grid, cudaStream_t st)
{
    het_mixed_hm_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}

template <int G, int BLOCK>
cudaError_t launch_het_mixed_pt(const HetLaunch& L, int grid, cudaStream_t st)
{
    if constexpr (BLOCK % 64 == 0)
        het_mixed_pt_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    else
        het_mixed_pt_kernel_capped<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}
}  // namespace

namespace mbh {
HetKernel het_kernel_mixed(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return {&launch_het_mixed<g, b>, het_mixed_fn<g, b>()};
    MBH_CASE(1, 64) MBH_CASE(1, 128) MBH_CASE(1, 256)
    MBH_CASE(2, 32) MBH_CASE(2, 64) MBH_CASE(2, 128) MBH_CASE(2, 256)
    MBH_CASE(4, 32) MBH_CASE(4, 64) MBH_CASE(4, 96) MBH_CASE(4, 128) MBH_CASE(4, 160) MBH_CASE(4, 224)
    MBH_CASE(4, 256)
    MBH_CASE(8, 64) MBH_CASE(8, 96) MBH_CASE(8, 128) MBH_CASE(8, 160) MBH_CASE(8, 224) MBH_CASE(8, 256)
    MBH_CASE(16, 64) MBH_CASE(16, 128) MBH_CASE(16, 224) MBH_CASE(16, 256)
    MBH_CASE(32, 64) MBH_CASE(32, 128) MBH_CASE(32, 256)
#undef MBH_CASE
    return {nullptr, nullptr};
}
}  // namespace mbh

namespace mbh {
HetKernel het_kernel_mixed_hm(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return {&launch_het_mixed_hm<g, b>, (const void*)&het_mixed_hm_kernel<g, b>};
    MBH_CASE(1, 64) MBH_CASE(1, 128) MBH_CASE(1, 256)
    MBH_CASE(2, 64) MBH_CASE(2, 128) MBH_CASE(2, 256)
    MBH_CASE(4, 64) MBH_CASE(4, 128) MBH_CASE(4, 256)
    MBH_CASE(8, 64) MBH_CASE(8, 128) MBH_CASE(8, 256)
    MBH_CASE(16, 64) MBH_CASE(16, 128) MBH_CASE(16, 256)
    MBH_CASE(32, 64) MBH_CASE(32, 128) MBH_CASE(32, 256)
#undef MBH_CASE
    return {nullptr, nullptr};
}
}  // namespace mbh

namespace mbh {
HetKernel het_kernel_mixed_pt(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return {&launch_het_mixed_pt<g, b>, het_mixed_pt_fn<g, b>()};
    MBH_CASE(1, 64) MBH_CASE(1, 128) MBH_CASE(1, 256)
    MBH_CASE(2, 32) MBH_CASE(2, 64) MBH_CASE(2, 128) MBH_CASE(2, 256)
    MBH_CASE(4, 32) MBH_CASE(4, 64) MBH_CASE(4, 96) MBH_CASE(4, 128) MBH_CASE(4, 160) MBH_CASE(4, 224)
    MBH_CASE(4, 256)
    MBH_CASE(8, 64) MBH_CASE(8, 96) MBH_CASE(8, 128) MBH_CASE(8, 160) MBH_CASE(8, 224) MBH_CASE(8, 256)
    MBH_CASE(16, 64) MBH_CASE(16, 128) MBH_CASE(16, 224) MBH_CASE(16, 256)
    MBH_CASE(32, 64) MBH_CASE(32, 128) MBH_CASE(32, 256)
#undef MBH_CASE
    return {nullptr, nullptr};
}
}  // namespace mbh

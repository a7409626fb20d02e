// Heterodyned likelihood in extended (double-float) precision, the MBH_MIXED path for (2,2)
// references (Katz, arXiv:2111.01064, Sec. II B, Eqs. 10-19; the batched evaluations of
// Sec. III B-C).
//
// Why the ratio is formed relative to the reference.  lnL = -1/2 <d - h|d - h> + const has, for
// a walker far from the data, a gradient of size ~<h|h> with respect to h: a relative error eps
// of the edge values r = h/h0 reaches lnL as ~<h|h> eps / sqrt(N_eff) (N_eff ~ 70-80 bins carry
// the weight of log-spaced bins).  At SNR 1000 (<h|h> = 1e6) |dlnL| <= 1e-3 for every walker of
// a batch needs eps <~ 1.5e-9 per edge, ~25 times below the float32 rounding of a response
// chain, and below what even a double-float phase Phi ~ 1e6 rad keeps (~5e-9 rad).  So no large
// quantity is formed at all: per walker, in float64, the coefficients of the *differences* to
// the reference are computed once,
//   Psi_PN(f) - Psi_PN,0(f) = sum_k D_k v0^{k-5} + ln v0 (Dl5 + Dl6 v0),
//   t(f) - t0(f)           = v0^{-8} sum_k E_k v0^k + v0^{-2} El6 ln v0 + dT0,
// (v = s v0 with s = (M/M0)^{1/3}, v0 = (pi M0 f)^{1/3} of the reference, so every power of v
// is a power of v0 times a walker constant), and the per-edge evaluation, in double-float on
// the float32 pipe, only ever handles the (small) differences: the phase difference
//   dPhi = f (C1 + 2 pi (AU/c) [k.c(t) - k0.c(t0)]) + dPsi_PN,
// the orbit at t = t0(f) + dt from the reference's angle alpha0(f) and the increment 2 pi dt/yr,
// the amplitude ratio R exp(-f^2 (1/fc^2 - 1/fc0^2)) (f^{-7/6} cancels), and the raw transfer of
// the walker, which the edge record's G_c = K_c/T0_c (float64, from the reference's transfer at
// alpha0(f) and the frequency-only factors K_c) turns into the response ratio.  All of these
// vanish (or are exactly 1) at the reference itself.  Then
//   delta_c = r_c - 1 = T_c (A e^{-i dPhi} G_c) - 1,   A = R e^u,
// and the contraction of Eqs. 14 and 17 is regrouped per edge (each edge's delta meets the
// summary data of its two bins through five double-float weights per channel; the bin's cross
// term needs the neighbouring edge's delta) and accumulated in double-float.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mbh_dfx.cuh"
#include "mbh_internal.cuh"
#include "mbh_mixed.cuh"
#include "mbh_model.cuh"
#include "mbh_pt.cuh"

using namespace mbh;

namespace mbh {

// sin(k pi/16), cos(k pi/16) - 1 for k = 0..16 (40-digit values, rounded to float64)
__device__ const double kSinTabD[17][2] = {
    {0.0, 0.0},
    {0.1950903220161282678482849, -0.01921471959676955087381776},
    {0.38268343236508977172846, -0.07612046748871324387181681},
    {0.5555702330196022247428308, -0.1685303876974547629212116},
    {0.7071067811865475244008444, -0.2928932188134524755991556},
    {0.8314696123025452370787884, -0.4444297669803977752571692},
    {0.9238795325112867561281832, -0.61731656763491022827154},
    {0.9807852804032304491261822, -0.8049096779838717321517151},
    {1.0, -1.0},
    {0.9807852804032304491261822, -1.195090322016128267848285},
    {0.9238795325112867561281832, -1.38268343236508977172846},
    {0.8314696123025452370787884, -1.555570233019602224742831},
    {0.7071067811865475244008444, -1.707106781186547524400844},
    {0.5555702330196022247428308, -1.831469612302545237078788},
    {0.38268343236508977172846, -1.923879532511286756128183},
    {0.1950903220161282678482849, -1.980785280403230449126182},
    {0.0, -2.0},
};

__device__ __forceinline__ f2 split_rn(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// Per-edge precision.  On an edge that takes the float32 ratio (the float32-ratio path's
// edge_delta_mixed: double-float phase, float32 response and ratio) delta is off by at most
// kF32EdgeError for |delta| <= kDeltaMax; with S_e >= |d lnL / d delta_e| the float32 edges add
// at most kF32EdgeError sum S_e <= kF32Budget to |dlnL|.  kF32EdgeError is ten times the largest
// error per unit of sensitivity that the float32 ratio shows with every edge in float32 (its
// batch maximum |dlnL| over sum S_e: 1.4e-8 to 2.8e-8 on sources of SNR 122 to 1000, whose
// walkers reach |delta| ~ 4).  The float32 error grows with |1 + delta| and the sensitivity with
// |delta|: a walker's float32 value is kept while every channel has |delta| <= kDeltaF32Max,
// where the product is at most 18 times its value at |delta| = 4 (5e-7 per unit of S_e, so the
// float32 edges add at most 5e-7 kF32Budget / kF32EdgeError = 5e-4 to |dlnL|, the double-float
// edges ~1e-4); beyond that the edge takes the double-float chain.  (A single float32 edge at the
// top of a band has shown 2e-7 per unit of S_e on a source drawn at random.)  With higher modes the float32 terms are the modes' shares u_g = h0_g/h0 of the
// reference, so near a zero of h0 (modes that cancel) the error grows by kappa = sum |u_g|:
// the selection weighs S_e by kappa_e.  Edges are chosen in aligned groups of kF32Group: with
// four threads per walker (the default) a group is one round of a warp's edges, so no warp
// runs both paths for one round.
constexpr double kDeltaMax = 3.0;
constexpr double kF32EdgeError = 3e-7;
constexpr double kF32Budget = 3e-4;
constexpr float kDeltaF32Max = 16.0f;
constexpr int kF32Group = 4;

__device__ __forceinline__ void load_sintab(SinTab& tab)
{
    for (int k = threadIdx.x; k < 17; k += blockDim.x) {
        const f2 s = split_rn(kSinTabD[k][0]), c = split_rn(kSinTabD[k][1]);
        tab.v[k] = make_float4(s.hi, s.lo, c.hi, c.lo);
    }
}

// v and ln v at f_max: pi M f_max = 0.05 pi sqrt(5/12) for every mass (f_max = f_c sqrt(5/12),
// f_c = 0.05/M), so v(f_max), ln v(f_max), v^-5 and v^-8 are constants (40-digit values).
constexpr double kXVm = 0.4663064457284195;
constexpr double kXLnVm = -0.7629122521271803;
constexpr double kXVm5Inv = 45.35685218040481;
constexpr double kXVm8Inv = 447.3306440422728;

// float64 quantities of one parameter vector (Sec. II A parameter derivation): the one
// derivation used for the reference and for the walkers, so that their differences vanish
// exactly for the reference itself.
__device__ inline void xderive(const double* __restrict__ theta, int64_t W, int64_t i, XDer& x)
{
    const double mt = theta[kMT * W + i], q = theta[kQ * W + i];
    const double a1 = theta[kA1 * W + i], a2 = theta[kA2 * W + i];
    const double tref = theta[kTref * W + i];
    const double lam = theta[kLam * W + i], bet = theta[kBeta * W + i];
    const double dl = theta[kDL * W + i], phi = theta[kPhi * W + i];
    const double iota = theta[kIota * W + i], pol = theta[kPsi * W + i];
    const double opq = 1.0 + q;
    const double M = mt * kMsunSec;
    const double dist = dl * (1e9 * kParsec / kClight);
    const double x1 = 1.0 / opq, x2 = q * x1;
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
    const double pre = 3.0 / (128.0 * eta), dpre = pre * (kPi / 3.0) * M;
    double c[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        c[k] = pre * al[k];
        d[k] = dpre * ((k - 5) * al[k]);
    }
    d[5] += dpre * alog5;
    d[6] += dpre * alog6;
    const double cl5 = pre * alog5, cl6 = pre * alog6, dl6 = dpre * alog6;
    double P = c[7], Q = d[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        P = fma(P, kXVm, c[k]);
        Q = fma(Q, kXVm, d[k]);
    }
    constexpr double vm5 = kXVm * kXVm * kXVm * kXVm * kXVm, vm6 = vm5 * kXVm;
    const double psi_max = (P + kXLnVm * (cl5 * vm5 + cl6 * vm6)) * kXVm5Inv;
    const double dpsi_max = (Q + kXLnVm * dl6 * vm6) * kXVm8Inv;
    const double fmax = 0.05 * 0.6454972243679028 / M;   // f_c sqrt(5/12)
    x.mt = mt;
    x.eta = eta;
    x.dist = dist;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x.c[k] = c[k];
        x.d[k] = d[k] * kInvTwoPi;
    }
    x.c[5] += fmax * dpsi_max - psi_max;   // the t_ref/f_max pinning's constant
    x.cl5 = cl5;
    x.cl6 = cl6;
    x.dl6 = dl6 * kInvTwoPi;
    x.t0 = tref - dpsi_max * kInvTwoPi;
    x.c1 = kTwoPi * tref - dpsi_max;
    x.fcut = 0.2 / M;
    x.ifc2 = 400.0 * M * M;
    double sl, cl, sb, cbt, s2p, c2p, s2f, c2f;
    sincos(lam, &sl, &cl);
    sincos(bet, &sb, &cbt);
    sincos(2.0 * pol, &s2p, &c2p);
    sincos(2.0 * phi, &s2f, &c2f);
    x.kx = kTwoPi * kAUSec * (-cbt * cl);
    x.ky = kTwoPi * kAUSec * (-cbt * sl);
    constexpr double isq3 = 0.57735026918962576451;
    x.k3[0] = -cbt * cl * isq3;
    x.k3[1] = -cbt * sl * isq3;
    x.k3[2] = -sb * isq3;
    x.eu[0] = sl * isq3;
    x.eu[1] = -cl * isq3;
    x.ev[0] = -sb * cl * isq3;
    x.ev[1] = -sb * sl * isq3;
    x.ev[2] = cbt * isq3;
    const double ylm = 0.15769578262626002 /* sqrt(5/(64 pi)) */;
    const double ci = cos(iota);
    const double ap = ylm * (1.0 + ci * ci), ac = 2.0 * ylm * ci;
    // K+ = ap e^{2i phi}, Kx = i ac e^{2i phi}; Ga = cos2psi K+ - sin2psi Kx, Gb = sin2psi K+ + cos2psi Kx
    x.G[0] = c2p * ap * c2f + s2p * ac * s2f;
    x.G[1] = c2p * ap * s2f - s2p * ac * c2f;
    x.G[2] = s2p * ap * c2f - c2p * ac * s2f;
    x.G[3] = s2p * ap * s2f + c2p * ac * c2f;
}

// Walker constants relative to the reference (double-float, shared memory).
struct XWalker {
    f2 D[8], Dl5, Dl6;   // phase difference coefficients (D[1] = 0)
    f2 E[8], El6, dT0;   // time difference coefficients
    f2 C1;               // coefficient of f: 2 pi (t_ref - t_ref0) - (psi'_max - psi'_max,0)
    f2 dkx, dky, kx, ky; // orbit phase: 2 pi AU/c (k - k0) and k of the walker (in-plane)
    f2 fcut, R, difc2;   // f_cut; amplitude ratio; 1/fc^2 - 1/fc0^2
    f2 k3[3], eu[2], ev[3], Ga[2], Gb[2];   // response constants (as the float32 path)
    f2 s;                // (M/M0)^{1/3}: v = s v0 (the higher modes' v^{p_lm})
};

// Higher modes: the walker's per-mode polarisation factors rotated by 2 psi, (Ga, Gb) as for the
// (2,2) mode, folded with H_lm's constant and sqrt(2/m) (the float64 model's hm_setup).
struct XWalkerHM {
    f2 G[kHmModes][4];   // Ga (re, im), Gb (re, im)
};

__device__ inline void xwalker_setup_hm(const double* __restrict__ theta, int64_t W, int64_t i, XWalkerHM& h)
{
    const double q = theta[kQ * W + i], iota = theta[kIota * W + i], phi = theta[kPhi * W + i];
    const double pol = theta[kPsi * W + i];
    Walker tmp;
    hm_setup(tmp, q, iota, phi);
    double s2p, c2p;
    sincos(2.0 * pol, &s2p, &c2p);
#pragma unroll
    for (int b = 0; b < kHmModes; ++b)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const double kp = tmp.hk[b][j], kc = tmp.hk[b][2 + j];
            h.G[b][j] = split_rn(c2p * kp - s2p * kc);
            h.G[b][2 + j] = split_rn(s2p * kp + c2p * kc);
        }
}

__device__ inline void xwalker_setup(const double* __restrict__ theta, int64_t W, int64_t i,
                                     const XDer& r, XWalker& o)
{
    XDer w;
    xderive(theta, W, i, w);
    const double rm = w.mt / r.mt;
    const double s = w.mt == r.mt ? 1.0 : cbrt(rm);
    const double ls = w.mt == r.mt ? 0.0 : log(rm) * (1.0 / 3.0);
    const double is = 1.0 / s;
    double sp[16];   // s^{k}, k = -8..7, at sp[k + 8]
    sp[8] = 1.0;
    for (int k = 1; k < 8; ++k) sp[8 + k] = sp[7 + k] * s;
    for (int k = 1; k <= 8; ++k) sp[8 - k] = sp[9 - k] * is;
    double D[8], E[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        D[k] = w.c[k] * sp[8 + k - 5] - r.c[k];
        E[k] = w.d[k] * sp[k] - r.d[k];   // s^{k - 8}
    }
    D[5] += w.cl5 * ls;
    D[6] += w.cl6 * s * ls;
    E[6] += w.dl6 * sp[6] * ls;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        o.D[k] = split_rn(D[k]);
        o.E[k] = split_rn(E[k]);
    }
    o.Dl5 = split_rn(w.cl5 - r.cl5);
    o.Dl6 = split_rn(w.cl6 * s - r.cl6);
    o.El6 = split_rn(w.dl6 * sp[6] - r.dl6);
    o.dT0 = split_rn(w.t0 - r.t0);
    o.C1 = split_rn(w.c1 - r.c1);
    o.dkx = split_rn(w.kx - r.kx);
    o.dky = split_rn(w.ky - r.ky);
    o.kx = split_rn(w.kx);
    o.ky = split_rn(w.ky);
    o.fcut = split_rn(w.fcut);
    // A(f) = sqrt(2 pi/3) pi^{-2/3} M^{5/6} eta^{1/2} f^{-7/6} exp(-(f/f_c)^2) / D: the ratio of
    // the f-independent factors is s^{5/2} (eta/eta0)^{1/2} D0/D
    o.R = split_rn(s * s * sqrt(s * w.eta / r.eta) * (r.dist / w.dist));
    o.difc2 = split_rn(w.ifc2 - r.ifc2);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.k3[j] = split_rn(w.k3[j]);
        o.ev[j] = split_rn(w.ev[j]);
    }
    o.eu[0] = split_rn(w.eu[0]);
    o.eu[1] = split_rn(w.eu[1]);
    o.Ga[0] = split_rn(w.G[0]);
    o.Ga[1] = split_rn(w.G[1]);
    o.Gb[0] = split_rn(w.G[2]);
    o.Gb[1] = split_rn(w.G[3]);
    o.s = split_rn(s);
}

// The per-arm body (three times per edge) and the double-float sine/cosine (four times per
// edge) come inlined (kInl, the (2,2) kernel: 2.4 % faster) or compiled once and called (the
// higher-mode kernel, whose loop holds four mode groups and the float32 path: inlined there,
// its instruction fetch stalls the warps and it runs 22 % slower).

constexpr f2 kH3 = df_const(0.8660254037844386467637231707529361835);   // sqrt3/2
constexpr f2 kH3q = df_const(0.8660254037844386467637231707529361835 / 4.0);   // sqrt3/8
constexpr f2 kH3x3q = df_const(0.8660254037844386467637231707529361835 * 0.75);   // 3 sqrt3/8
constexpr f2 kOrbRate = df_const(6.283185307179586476925286766559005768 / 31557600.0);   // 2 pi / yr

// sin(x(1 - kn)) and sinc(x(1 + kn)) - sinc(x(1 - kn)) of one arm (the one-link sinc factors
// of the float32 path's transfer).  Below x = 0.3: sinc(b) = 1 - b^2/6 + b^4 (...) with the b^4
// tail in float32 (< 1.1e-3, rounding < 7e-11), and the difference as 4 x^2 kn (-1/6 + S) with
// S = sum_{j>=2} (-1)^j P_j/(2j+1)! (P_1 = 1, P_{j+1} = a^2 P_j + b^{2j}, a = x(1 + kn),
// b = x(1 - kn)) in float32 (|S| < 6e-3); above, both sincs in double-float.
__device__ __forceinline__ void arm_sincs(f2 x, f2 kn, const SinTab& tab, f2& sm, f2& sd)
{
    const f2 b = dd_mul_lazy(x, dd_add_f_lazy({-kn.hi, -kn.lo}, 1.0f));
    if (x.hi < 0.3f) {
        const f2 b2 = dd_sqr_lazy(b);
        const float z = b2.hi;
        const float tail = z * z * fmaf(z, fmaf(z, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f);
        sm = dd_add_f_lazy(dd_add_f_lazy(dd_mul_lazy(b2, kSc1), tail), 1.0f);
        const float xa = x.hi * (1.0f + kn.hi), a2 = xa * xa;
        float P = 1.0f, bp = 1.0f, S = 0.0f, sg = 1.0f;
        constexpr float inv_fact[4] = {1.0f / 120.0f, 1.0f / 5040.0f, 1.0f / 362880.0f, 1.0f / 39916800.0f};
#pragma unroll
        for (int j = 0; j < 4; ++j) {   // P_{j+2} and the terms j + 2 = 2..5
            bp *= z;
            P = fmaf(a2, P, bp);
            S = fmaf(sg * P, inv_fact[j], S);
            sg = -sg;
        }
        const f2 k4 = dd_scale(dd_mul_lazy(dd_sqr_lazy(x), kn), 4.0f);
        sd = dd_add_f_lazy(dd_mul_lazy(k4, kSc1), k4.hi * S);
    } else {
        const f2 a = dd_mul_lazy(x, dd_add_f_lazy(kn, 1.0f));
        sm = dd_sinc(b, tab);
        sd = dd_sub_lazy(dd_sinc(a, tab), sm);
    }
}

struct SinCos {
    f2 s, cm1;
};

__device__ __forceinline__ SinCos sincos_df_body(f2 x, const SinTab& tab)
{
    SinCos r;
    dd_sincos_any(x, tab, r.s, r.cm1);
    return r;
}

__device__ __noinline__ SinCos sincos_df_call(f2 x, const SinTab& tab) { return sincos_df_body(x, tab); }

template <bool kInl>
__device__ __forceinline__ SinCos sincos_df(f2 x, const SinTab& tab)
{
    if constexpr (kInl)
        return sincos_df_body(x, tab);
    else
        return sincos_df_call(x, tab);
}

struct ArmOut {
    c2f yf, z;
};

// One arm (spacecraft i -> j, third spacecraft m) of the raw transfer: arm vector d = u_j - u_i,
// kn = k.n, the polarisation response a Ga + b Gb, g = i e^{i q_m} F and the one-link sinc
// factors: yf = g sinc(x(1 - kn)), z = g [sinc(x(1 + kn)) - sinc(x(1 - kn))].
__device__ __forceinline__ ArmOut arm_df_body(const XWalker& w, const f2* Ga, const f2* Gb, f2 x, f2 d0, f2 d1,
                                              f2 d2, f2 kn, c2f Em, const SinTab& tab)
{
    const f2 un = dd_add_lazy(dd_mul_lazy(w.eu[0], d0), dd_mul_lazy(w.eu[1], d1));
    const f2 vn = dd_add_lazy(dd_add_lazy(dd_mul_lazy(w.ev[0], d0), dd_mul_lazy(w.ev[1], d1)),
                              dd_mul_lazy(w.ev[2], d2));
    const f2 pa = dd_sub_lazy(dd_sqr_lazy(un), dd_sqr_lazy(vn));
    const f2 pb = dd_scale(dd_mul_lazy(un, vn), 2.0f);
    const c2f F = {dd_add_lazy(dd_mul_lazy(pa, Ga[0]), dd_mul_lazy(pb, Gb[0])),
                   dd_add_lazy(dd_mul_lazy(pa, Ga[1]), dd_mul_lazy(pb, Gb[1]))};
    const c2f eF = cd_mul(Em, F);
    const c2f g = {{-eF.im.hi, -eF.im.lo}, eF.re};   // i e^{i q_m} F
    f2 sm, sd;
    arm_sincs(x, kn, tab, sm, sd);
    return {cd_mul_r(g, sm), cd_mul_r(g, sd)};
}

__device__ __noinline__ ArmOut arm_df_call(const XWalker& w, const f2* Ga, const f2* Gb, f2 x, f2 d0, f2 d1, f2 d2,
                                           f2 kn, c2f Em, const SinTab& tab)
{
    return arm_df_body(w, Ga, Gb, x, d0, d1, d2, kn, Em, tab);
}

template <bool kInl>
__device__ __forceinline__ ArmOut arm_df(const XWalker& w, const f2* Ga, const f2* Gb, f2 x, f2 d0, f2 d1, f2 d2,
                                         f2 kn, c2f Em, const SinTab& tab)
{
    if constexpr (kInl)
        return arm_df_body(w, Ga, Gb, x, d0, d1, d2, kn, Em, tab);
    else
        return arm_df_call(w, Ga, Gb, x, d0, d1, d2, kn, Em, tab);
}

// Raw transfer of the walker at orbit angle (sa, ca): the construction of the float32 path's
// transfer_f32<raw> (spacecraft offsets u_i in units of L/sqrt3, arm phases x - q_m with
// e^{i q_m}, q_m = x (k/sqrt3).u_m, polarisation response a Ga + b Gb, one-link sinc factors,
// first-generation TDI with D = e^{-2ix} = (c2, -s2)) in double-float:
//   T_A = P_A + D Q_A, T_E = P_E + D Q_E, T_T = z0 + z1 + z2 with, per arm, yf = g sinc(x(1-kn))
//   and z = g [sinc(x(1+kn)) - sinc(x(1-kn))],
//   P_A = U - z0, Q_A = U - z1, U = 2 yf2 + z2 - yf1 - yf0,
//   P_E = V + z0 + z2 - 2 z1, Q_E = V + 2 z0 - z2 - z1, V = 3 (yf0 - yf1).
// T is linear in (Ga, Gb): the mode factors (the walker's (2,2) ones, or a higher-mode group's
// sum), here already multiplied by the amplitude and phase factor A e^{-i dPhi}.
template <bool kInl>
__device__ inline void transfer_df(const XWalker& w, const f2* Ga, const f2* Gb, f2 x, f2 s2, f2 c2, f2 sa, f2 ca,
                                   const SinTab& tab, c2f T[3])
{
    // spacecraft offsets from the double angle: with C = cos 2a, S = sin 2a, b_i = 2 pi i/3,
    //   u_i = ((cos(2a - b_i) - 3 cos b_i)/4, (sin(2a - b_i) - 3 sin b_i)/4, -h3 cos(a - b_i))
    const f2 S = dd_scale(dd_mul_lazy(sa, ca), 2.0f);
    const f2 C = dd_sub_lazy(dd_sqr_lazy(ca), dd_sqr_lazy(sa));
    const f2 hS = dd_mul_lazy(kH3q, S), hC = dd_mul_lazy(kH3q, C);   // (h3/4) S, (h3/4) C
    const f2 x0 = dd_add_f_lazy(dd_scale(C, -0.125f), 0.375f);       // (3 - C)/8
    const f2 y0 = dd_add_lazy(hC, kH3x3q);                            // (h3/4) C + 3 h3/4
    const f2 sq = dd_scale(S, -0.125f);                               // -S/8
    const f2 hca = dd_mul_lazy(kH3, ca), hca2 = dd_scale(hca, 0.5f), sa3 = dd_mul_f_lazy(sa, 0.75f);
    const f2 u[3][3] = {{dd_add_f_lazy(dd_scale(C, 0.25f), -0.75f), dd_scale(S, 0.25f), {-hca.hi, -hca.lo}},
                        {dd_add_lazy(x0, hS), dd_sub_lazy(sq, y0), dd_sub_lazy(hca2, sa3)},
                        {dd_sub_lazy(x0, hS), dd_add_lazy(sq, y0), dd_add_lazy(hca2, sa3)}};
    f2 kap[3];
#pragma unroll
    for (int m = 0; m < 2; ++m)
        kap[m] = dd_add_lazy(dd_add_lazy(dd_mul_lazy(w.k3[0], u[m][0]), dd_mul_lazy(w.k3[1], u[m][1])),
                             dd_mul_lazy(w.k3[2], u[m][2]));
    kap[2] = dd_add_lazy(kap[0], kap[1]);
    kap[2] = {-kap[2].hi, -kap[2].lo};
    c2f E[3];   // e^{i q_m}
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const SinCos q = sincos_df<kInl>(dd_mul_lazy(x, kap[m]), tab);
        E[m] = {dd_add_f_lazy(q.cm1, 1.0f), q.s};
    }
    const c2f e01 = cd_mul(E[0], E[1]);
    E[2] = {e01.re, {-e01.im.hi, -e01.im.lo}};
    c2f yf[3], z[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = a, j = (a + 1) % 3, m = (a + 2) % 3;
        f2 d[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] = dd_sub_lazy(u[j][q], u[i][q]);
        const ArmOut o = arm_df<kInl>(w, Ga, Gb, x, d[0], d[1], d[2], dd_sub_lazy(kap[j], kap[i]), E[m], tab);
        yf[a] = o.yf;
        z[a] = o.z;
    }
    const c2f U = cd_sub(cd_sub(cd_add(cd_scale(yf[2], 2.0f), z[2]), yf[1]), yf[0]);
    const c2f PA = cd_sub(U, z[0]), QA = cd_sub(U, z[1]);
    const c2f d01 = cd_sub(yf[0], yf[1]);
    const c2f V = cd_add(cd_scale(d01, 2.0f), d01);
    const c2f PE = cd_sub(cd_add(cd_add(V, z[0]), z[2]), cd_scale(z[1], 2.0f));
    const c2f QE = cd_sub(cd_sub(cd_add(V, cd_scale(z[0], 2.0f)), z[2]), z[1]);
    const c2f D = {c2, {-s2.hi, -s2.lo}};
    T[0] = cd_add(PA, cd_mul(D, QA));
    T[1] = cd_add(PE, cd_mul(D, QE));
    T[2] = cd_add(cd_add(z[0], z[1]), z[2]);
}

// One mode group's share of r = h/h0 at an edge (Sec. II B, Eq. 10), double-float: T_c G_c
// (c = A, E, T) with T_c the raw transfer of the mode factors times A e^{-i dPhi}, added to
// acc[c] (kAdd) or stored there; returns false, leaving acc unchanged, outside the walker's support (f2 > f_cut or t outside [0, t_obs]).  The group's modes share f2 = 2f/m,
// the phase chain (scaled by m/2), t(f2) and the orbit; the (2,2) mode alone is one group with
// m = 2.  v0, 1/v0, ln v0 are the reference's at f2; t0, (ca0, sa0) its time and orbit angle
// at f2; G4: the record's three G_c as float4 (re hi, re lo, im hi, im lo); Ga, Gb the mode
// factors (summed over the group's modes with their v^{p_lm}).
template <bool kAdd, bool kInl>
__device__ __forceinline__ bool group_term(const XWalker& w, const f2* Ga, const f2* Gb, f2 f, f2 fm, f2 v0, f2 iv0,
                                           f2 lnv0, float half_m, f2 t0, f2 ca0, f2 sa0, f2 x, f2 s2, f2 c2,
                                           const float4* G4, f2 tob, const SinTab& tab, c2f acc[3])
{
    // t(f2) - t0(f2) and the support test on t = t0 + dt, f2 <= f_cut
    f2 Q = w.E[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) Q = dd_fma_lazy(Q, v0, w.E[k]);
    const f2 iv2 = dd_sqr_lazy(iv0), iv4 = dd_sqr_lazy(iv2), iv8 = dd_sqr_lazy(iv4);
    const f2 dt = dd_add_lazy(dd_add_lazy(dd_mul_lazy(Q, iv8), dd_mul_lazy(dd_mul_lazy(w.El6, lnv0), iv2)), w.dT0);
    const f2 t = dd_add(t0, dd_norm(dt));
    if (!(dd_le(fm, w.fcut) && !dd_lt0(t) && dd_le(t, tob))) return false;
    // orbit angle alpha = alpha0 + 2 pi dt / yr
    const SinCos oa = sincos_df<kInl>(dd_mul_lazy(dt, kOrbRate), tab);
    const f2 sD = oa.s, cD = oa.cm1;
    const f2 sa = dd_add_lazy(sa0, dd_add_lazy(dd_mul_lazy(sa0, cD), dd_mul_lazy(ca0, sD)));
    const f2 ca = dd_add_lazy(ca0, dd_sub_lazy(dd_mul_lazy(ca0, cD), dd_mul_lazy(sa0, sD)));
    // 2 pi AU/c [k.c(t) - k0.c(t0)] = dk.c(t0) + (cos da - 1) k.c(t0) + sin da (k x c(t0))_z
    const f2 kc0 = dd_add_lazy(dd_mul_lazy(w.kx, ca0), dd_mul_lazy(w.ky, sa0));
    const f2 ks0 = dd_sub_lazy(dd_mul_lazy(w.ky, ca0), dd_mul_lazy(w.kx, sa0));
    const f2 dorb = dd_add_lazy(dd_add_lazy(dd_mul_lazy(w.dkx, ca0), dd_mul_lazy(w.dky, sa0)),
                                dd_add_lazy(dd_mul_lazy(cD, kc0), dd_mul_lazy(sD, ks0)));
    // Psi_PN - Psi_PN,0 = sum_k D_k v0^{k-5} + ln v0 (Dl5 + Dl6 v0) at f2
    f2 N = dd_mul_lazy(w.D[0], iv0);
#pragma unroll
    for (int k = 2; k <= 5; ++k) N = dd_fma_lazy(N, iv0, w.D[k]);
    const f2 Pp = dd_mul_lazy(dd_fma_lazy(w.D[7], v0, w.D[6]), v0);
    const f2 L = dd_mul_lazy(lnv0, dd_fma_lazy(w.Dl6, v0, w.Dl5));
    // dPhi = f (C1 + dorb) + (m/2) dPsi_PN(f2)  (the f2 t_ref terms of (m/2) Phi_22(f2) are f C1)
    const f2 dpsi = dd_mul_f_lazy(dd_add_lazy(dd_add_lazy(N, Pp), L), half_m);
    const f2 dphi = dd_norm(dd_add_lazy(dd_mul_lazy(f, dd_add_lazy(w.C1, dorb)), dpsi));
    const SinCos ph = sincos_df<kInl>(dphi, tab);
    // amplitude ratio A = R exp(-f2^2 (1/fc^2 - 1/fc0^2)), folded with e^{-i dPhi}:
    // Z = A e^{-i dPhi} = A + A (e^{-i dPhi} - 1), and Z into the mode factors
    const f2 u = dd_mul_lazy(dd_sqr_lazy(fm), w.difc2);
    const f2 A = dd_mul_lazy(w.R, dd_exp({-u.hi, -u.lo}));
    const c2f Z = {dd_add_lazy(A, dd_mul_lazy(A, ph.cm1)), dd_mul_lazy(A, {-ph.s.hi, -ph.s.lo})};
    const c2f za = cd_mul(Z, {Ga[0], Ga[1]}), zb = cd_mul(Z, {Gb[0], Gb[1]});
    const f2 zGa[2] = {za.re, za.im}, zGb[2] = {zb.re, zb.im};
    c2f T[3];
    transfer_df<kInl>(w, zGa, zGb, x, s2, c2, sa, ca, tab, T);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 g = G4[c];
        const c2f p = cd_mul(T[c], {{g.x, g.y}, {g.z, g.w}});
        acc[c] = kAdd ? cd_add(acc[c], p) : p;
    }
    return true;
}

// delta = r - 1 of one walker at one edge record of a (2,2) reference (Sec. II B, Eq. 10),
// double-float; -1 where the walker's template or the reference's is zero.
__device__ __forceinline__ void edge_delta_x(const XWalker& w, const XEdge* __restrict__ pe, f2 tob,
                                             const SinTab& tab, c2f dl[3])
{
    const float4* p4 = reinterpret_cast<const float4*>(pe);
    const float4 r0 = p4[0], r1 = p4[1], r2 = p4[2], r3 = p4[3], r4 = p4[4];
    const f2 f = {r0.x, r0.y}, v0 = {r0.z, r0.w}, iv0 = {r1.x, r1.y}, lnv0 = {r1.z, r1.w};
    const f2 t0 = {r2.x, r2.y}, ca0 = {r2.z, r2.w}, sa0 = {r3.x, r3.y}, x = {r3.z, r3.w};
    const f2 s2 = {r4.x, r4.y}, c2 = {r4.z, r4.w};
    c2f acc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    if (!group_term<false, true>(w, w.Ga, w.Gb, f, f, v0, iv0, lnv0, 1.0f, t0, ca0, sa0, x, s2, c2, p4 + 5, tob, tab, acc)) {
#pragma unroll
        for (int c = 0; c < 3; ++c) dl[c] = {{-1.0f, 0.0f}, {0.0f, 0.0f}};   // h = 0: r = 0
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) dl[c] = cd_norm({dd_add_f_lazy(acc[c].re, -1.0f), acc[c].im});
}

// Per group g = 0..3 (m = 2, 3, 4, 1): f2/f = 2/m, (2/m)^{1/3}, (m/2)^{1/3}, ln((2/m)^{1/3}), m/2
__constant__ float kGrpHalfM[4] = {1.0f, 1.5f, 2.0f, 0.5f};
__constant__ f2 kGrpR[4] = {df_const(1.0), df_const(2.0 / 3.0), df_const(0.5), df_const(2.0)};
__constant__ f2 kGrpR3[4] = {df_const(1.0), df_const(0.87358046473629952), df_const(0.79370052598409974),
                          df_const(1.2599210498948732)};
__constant__ f2 kGrpRm3[4] = {df_const(1.0), df_const(1.1447142425533319), df_const(1.2599210498948732),
                           df_const(0.79370052598409974)};
__constant__ f2 kGrpLn3[4] = {df_const(0.0), df_const(-0.13515503603605479), df_const(-0.23104906018664842),
                           df_const(0.23104906018664842)};

// delta = r - 1 of one walker at one edge of a higher-mode reference (Sec. II B, Eq. 10, with the
// template of Eq. 9 summed over the modes): r = sum over the reference's mode groups of the
// group's share (group_term), the group's mode factors summed with v^{p_lm} = (s v0(f2))^{p_lm}.
__device__ __forceinline__ void edge_delta_xhm(const XWalker& w, const XWalkerHM& wh, const XEdge* __restrict__ pe,
                                               const XGrp* __restrict__ pg, uint32_t modes, f2 tob,
                                               const SinTab& tab, c2f dl[3])
{
    const float4* p4 = reinterpret_cast<const float4*>(pe);
    const float4 r0 = p4[0], r1 = p4[1], r3 = p4[3], r4 = p4[4];
    const f2 f = {r0.x, r0.y}, v0 = {r0.z, r0.w}, iv0 = {r1.x, r1.y}, lnv0 = {r1.z, r1.w};
    const f2 x = {r3.z, r3.w}, s2 = {r4.x, r4.y}, c2 = {r4.z, r4.w};
    c2f acc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    bool any = false;
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
        const uint32_t gmask = modes & hm_group_mask(g);
        if (!gmask) continue;
        const float4* q4 = reinterpret_cast<const float4*>(pg + g);
        const float4 a = q4[0], b = q4[1];
        const f2 t0 = {a.x, a.y}, ca0 = {a.z, a.w}, sa0 = {b.x, b.y};
        const f2 v0m = dd_mul_lazy(v0, kGrpR3[g]), iv0m = dd_mul_lazy(iv0, kGrpRm3[g]);
        const f2 lnv0m = dd_add_lazy(lnv0, kGrpLn3[g]), fm = dd_norm(dd_mul_lazy(f, kGrpR[g]));
        // the group's mode factors: sum of v^{p_lm} (Ga, Gb)_lm, v = s v0(f2)
        const f2 vm = dd_mul_lazy(w.s, v0m);
        f2 G[4] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
        for (uint32_t bm = gmask; bm; bm &= bm - 1) {
            const int md = __ffs(bm) - 1;
            const int pw = hm_vpow(md);
            f2 vp = {1.0f, 0.0f};
            for (int j = 0; j < pw; ++j) vp = dd_mul_lazy(vp, vm);
#pragma unroll
            for (int j = 0; j < 4; ++j) G[j] = dd_add_lazy(G[j], dd_mul_lazy(vp, wh.G[md][j]));
        }
        // G4 of this group: float4 2, 3, 4 of the record are (G_A), (G_E), (G_T) after the 6
        // floats of t0, ca0, sa0 and 2 of padding
        any |= group_term<true, false>(w, &G[0], &G[2], f, fm, v0m, iv0m, lnv0m, kGrpHalfM[g], t0, ca0, sa0, x, s2, c2, q4 + 2,
                          tob, tab, acc);
    }
    if (!any) {
#pragma unroll
        for (int c = 0; c < 3; ++c) dl[c] = {{-1.0f, 0.0f}, {0.0f, 0.0f}};   // h = 0: r = 0
        return;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) dl[c] = cd_norm({dd_add_f_lazy(acc[c].re, -1.0f), acc[c].im});
}

// The edge's share of <d|h> and <h|h> (Eqs. 14 and 17 regrouped per edge, factor 4 included):
//   <d|h>: war Re delta + wai Im delta,
//   <h|h>: wbr Re delta + wq |delta|^2 + wc Re(delta_prev conj(delta)),
// with delta_prev the previous edge's (its bin's cross term; wc = 0 at edge 0).
__device__ __forceinline__ void contract_x(const XWeight* __restrict__ pw, const c2f dp[3], const c2f dl[3],
                                           f2& adh, f2& ahh)
{
    const float4* p4 = reinterpret_cast<const float4*>(pw);
    const float4 wc01 = p4[6], wc2 = p4[7];
    const f2 wc[3] = {{wc01.x, wc01.y}, {wc01.z, wc01.w}, {wc2.x, wc2.y}};
    f2 sdh = {0.0f, 0.0f}, shh = {0.0f, 0.0f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 a = p4[2 * c], b = p4[2 * c + 1];
        sdh = dd_add_lazy(sdh, dd_add_lazy(dd_mul_lazy({a.x, a.y}, dl[c].re), dd_mul_lazy({a.z, a.w}, dl[c].im)));
        const f2 m2 = dd_add_lazy(dd_sqr_lazy(dl[c].re), dd_sqr_lazy(dl[c].im));
        const f2 cr = dd_add_lazy(dd_mul_lazy(dp[c].re, dl[c].re), dd_mul_lazy(dp[c].im, dl[c].im));
        shh = dd_add_lazy(shh, dd_add_lazy(dd_add_lazy(dd_mul_lazy({b.x, b.y}, dl[c].re), dd_mul_lazy({b.z, b.w}, m2)),
                                           dd_mul_lazy(wc[c], cr)));
    }
    df_acc(adh, sdh);
    df_acc(ahh, shh);
}

// The float32 value of an edge is kept while every channel has |delta| <= kDeltaF32Max.
__device__ __forceinline__ bool f32_edge_small(const cf d[3])
{
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) ok &= d[c].re * d[c].re + d[c].im * d[c].im <= kDeltaF32Max * kDeltaF32Max;
    return ok;
}

// A float32-ratio edge value as double-float, with the rounding of the float32 amplitude
// factors removed: that rounding scales every float32 ratio of the walker alike (r' = r / fix,
// amp_fix), so delta = (1 + d) fix - 1 = d + eta (1 + d) with eta = fix - 1 (~1e-7).
__device__ __forceinline__ void f32_edge_df(const cf d[3], float eta, c2f dl[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c)
        dl[c] = {dd_add_f_lazy({d[c].re, 0.0f}, eta * (1.0f + d[c].re)), dd_add_f_lazy({d[c].im, 0.0f}, eta * d[c].im)};
}

// ------------------------------------------------------------------------------------------
// the kernel: layout and reductions as the float32 path's het_mixed_kernel (tiles of BLOCK/G
// walkers of one source, G threads per walker dealing the edges round-robin, the previous
// edge's delta from the neighbouring lane, lane sums reduced in a fixed order).  kPt: one
// sampler half step (Sec. III) in the same launch, as the float32-ratio het_mixed_pt_kernel:
// the walkers are the moving walkers' proposals (pt::propose_item in the set-up, kept in shared
// memory) and the epilogue applies the tempered acceptance test (pt::accept_test) instead of
// writing lnL.
// ------------------------------------------------------------------------------------------
template <int G, int BLOCK, bool kPt>
__device__ __forceinline__ void het_x_body(const HetLaunch& L)
{
    constexpr int WPB = BLOCK / G;
    constexpr int kSlot = (WPB + 31) / 32 * 32;
    constexpr int PW = kPt ? WPB : 1;
    __shared__ XWalker xw[WPB];
    __shared__ WalkerDF wsd[WPB];   // float32-ratio edges: the float32 path's walker constants
    __shared__ WalkerF wsf[WPB];
    __shared__ float eta32[WPB];    // and its amplitude rounding (f32_edge_df)
    __shared__ SinTab tab;
    __shared__ double ths[PW][pt::kPar];   // kPt: the proposals' theta (set-ups) and x (accepted)
    __shared__ double ys[PW][pt::kPar];
    __shared__ double facs[PW];
    __shared__ int32_t flags[PW];
    const int lw = threadIdx.x / G, lane = threadIdx.x % G;
    load_sintab(tab);
    for (int tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
        int s = 0;
        while (s + 1 < L.n_src && L.src[s + 1].tile_begin <= tile) ++s;
        const SrcDesc& S = L.src[s];
        const int64_t w0 = S.w_begin + (int64_t)(tile - S.tile_begin) * WPB;
        const bool active = w0 + lw < S.w_end;
        __syncthreads();
        if constexpr (kPt) {
            const pt::PtArgs& A = *static_cast<const pt::PtArgs*>(L.pt);
            for (int j = threadIdx.x; j < WPB; j += BLOCK)
                if (w0 + j < S.w_end) {
                    int32_t flag;
                    pt::propose_item(A, L.pt_half, (int32_t)(w0 + j), *A.step, ys[j], ths[j], facs[j], flag);
                    flags[j] = flag;
                }
            __syncthreads();
        }
        // the walkers' two set-ups (float64 chains bound by latency, not by the float64 pipe's
        // rate) on different warps where the block has them: slot t < WPB sets up walker t's
        // double-float constants, slot kSlot + t its float32-path constants (kSlot: WPB rounded
        // up to whole warps, so that no warp runs both chains one after the other)
        for (int t = threadIdx.x; t < 2 * kSlot; t += BLOCK) {
            const int j = t < kSlot ? t : t - kSlot;
            if (j >= WPB || w0 + j >= S.w_end) continue;
            const double* th = L.theta;   // the batch's theta, or the proposal in shared memory
            int64_t tw = L.W, ti = w0 + j;
            if constexpr (kPt) {
                th = &ths[j][0];
                tw = 1;
                ti = 0;
            }
            if (t < kSlot) {
                xwalker_setup(th, tw, ti, *S.mix.xder, xw[j]);
            } else if (S.mix.xn32 > 0) {
                walker_setup_mixed(th, tw, ti, wsd[j], wsf[j]);
                eta32[j] = (float)(amp_fix(wsf[j].eps_amp76, S.mix.amp_eps0) - 1.0);
            }
        }
        __syncthreads();
        const int E = S.E;
        const f2 tob = {S.tob_hi, S.tob_lo};
        f2 adh = {0.0f, 0.0f}, ahh = {0.0f, 0.0f};
        c2f carry[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) carry[c] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
        const int rounds = (E + 1 + G - 1) / G;
        for (int r = 0; r < rounds; ++r) {
            const int e = r * G + lane;
            c2f dl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) dl[c] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
            // (debug builds: the edge index against the source's logical range; a failed
            // check is recorded in the status word and the edge skipped)
            const bool ok = active && e <= E && MBH_IN_RANGE(L.status, e, (long long)S.E_check + 1, kKernHetX, s);
            if (ok) {
                bool done = false;
                if (S.mix.xw[e].v[30] != 0.0f) {   // low-weight edge: float32 ratio
                    cf d32[3];
                    edge_delta_mixed(wsd[lw], wsf[lw], S.mix.edge + e, tob, d32);
                    if (f32_edge_small(d32)) {
                        f32_edge_df(d32, eta32[lw], dl);
                        done = true;
                    }
                }
                if (!done) edge_delta_x(xw[lw], S.mix.xedge + e, tob, tab, dl);
            }
            c2f dp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dp[c].re.hi = __shfl_up_sync(0xffffffffu, dl[c].re.hi, 1, G);
                dp[c].re.lo = __shfl_up_sync(0xffffffffu, dl[c].re.lo, 1, G);
                dp[c].im.hi = __shfl_up_sync(0xffffffffu, dl[c].im.hi, 1, G);
                dp[c].im.lo = __shfl_up_sync(0xffffffffu, dl[c].im.lo, 1, G);
                if (lane == 0) dp[c] = carry[c];
                carry[c].re.hi = __shfl_sync(0xffffffffu, dl[c].re.hi, G - 1, G);
                carry[c].re.lo = __shfl_sync(0xffffffffu, dl[c].re.lo, G - 1, G);
                carry[c].im.hi = __shfl_sync(0xffffffffu, dl[c].im.hi, G - 1, G);
                carry[c].im.lo = __shfl_sync(0xffffffffu, dl[c].im.lo, G - 1, G);
            }
            if (ok) contract_x(S.mix.xw + e, dp, dl, adh, ahh);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const f2 odh = {__shfl_down_sync(0xffffffffu, adh.hi, o, G), __shfl_down_sync(0xffffffffu, adh.lo, o, G)};
            const f2 ohh = {__shfl_down_sync(0xffffffffu, ahh.hi, o, G), __shfl_down_sync(0xffffffffu, ahh.lo, o, G)};
            df_acc(adh, odh);
            df_acc(ahh, ohh);
        }
        if (lane == 0 && active) {
            const int64_t wi = w0 + lw;
            const double dh = S.mix.xsumA + df_to_double(adh);
            const double hh = S.mix.xsumB + df_to_double(ahh);
            const double lnl = -0.5 * (S.dd + hh - 2.0 * dh);
            if constexpr (kPt) {
                const pt::PtArgs& A = *static_cast<const pt::PtArgs*>(L.pt);
                int32_t col;
                int t, cb;
                const int32_t flag = flags[lw];
                const int kind = flag >> 1;
                const bool acc = pt::accept_test(A, L.pt_half, (int32_t)wi, lnl, facs[lw], flag, col, t, cb);
                atomicAdd(&A.counters[cb + t * 4 + kind], 1ull);
                if (acc) {
                    atomicAdd(&A.counters[cb + 4 * A.T + t * 4 + kind], 1ull);
                    const int64_t N = (int64_t)A.n_ens * A.T * A.W;
#pragma unroll
                    for (int p = 0; p < pt::kPar; ++p) A.x[p * N + col] = ys[lw][p];
                    A.out[col] = lnl;
                    A.out[N + col] = dh;
                    A.out[2 * N + col] = hh;
                }
            } else {
                L.out[wi] = lnl;
                L.out[L.W + wi] = dh;
                L.out[2 * L.W + wi] = hh;
            }
        }
    }
}

template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK) het_x_kernel(const __grid_constant__ HetLaunch L)
{
    het_x_body<G, BLOCK, false>(L);
}

// one fused sampler half step (blocks of at most 32 walkers: the proposals' shared arrays)
template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK) het_x_pt_kernel(const __grid_constant__ HetLaunch L)
{
    het_x_body<G, BLOCK, true>(L);
}

// Higher-mode references (Sec. II B with the template of Eq. 9): the layout of het_x_kernel, the
// edge value from edge_delta_xhm (double-float) or, on the edges flagged for it, the float32
// ratio of the float32 higher-mode path (edge_delta_mixed_hm).
template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK) het_xhm_kernel(const __grid_constant__ HetLaunch L)
{
    constexpr int WPB = BLOCK / G;
    constexpr int kSlot = (WPB + 31) / 32 * 32;
    __shared__ XWalker xw[WPB];
    __shared__ XWalkerHM xh[WPB];
    __shared__ WalkerDF wsd[WPB];   // float32-ratio edges: the float32 path's walker constants
    __shared__ WalkerF wsf[WPB];
    __shared__ WalkerHMF wsh[WPB];
    __shared__ float eta32[WPB];
    __shared__ SinTab tab;
    const int lw = threadIdx.x / G, lane = threadIdx.x % G;
    load_sintab(tab);
    for (int tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
        int s = 0;
        while (s + 1 < L.n_src && L.src[s + 1].tile_begin <= tile) ++s;
        const SrcDesc& S = L.src[s];
        const int64_t w0 = S.w_begin + (int64_t)(tile - S.tile_begin) * WPB;
        const bool active = w0 + lw < S.w_end;
        __syncthreads();
        // the walkers' four set-ups on different warps where the block has them (slot
        // k kSlot + t: set-up k of walker t, kSlot = WPB rounded up to whole warps)
        for (int t = threadIdx.x; t < 4 * kSlot; t += BLOCK) {
            const int k = t / kSlot, j = t - k * kSlot;
            if (j >= WPB || w0 + j >= S.w_end) continue;
            if (k == 0) {
                xwalker_setup(L.theta, L.W, w0 + j, *S.mix.xder, xw[j]);
            } else if (k == 1) {
                xwalker_setup_hm(L.theta, L.W, w0 + j, xh[j]);
            } else if (S.mix.xn32 > 0) {
                if (k == 2) {
                    walker_setup_mixed(L.theta, L.W, w0 + j, wsd[j], wsf[j]);
                    eta32[j] = (float)(amp_fix(wsf[j].eps_amp76, S.mix.amp_eps0) - 1.0);
                } else {
                    walker_setup_hm(L.theta, L.W, w0 + j, wsh[j]);
                }
            }
        }
        __syncthreads();
        const int E = S.E;
        const f2 tob = {S.tob_hi, S.tob_lo};
        f2 adh = {0.0f, 0.0f}, ahh = {0.0f, 0.0f};
        c2f carry[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) carry[c] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
        const int rounds = (E + 1 + G - 1) / G;
        for (int r = 0; r < rounds; ++r) {
            const int e = r * G + lane;
            c2f dl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) dl[c] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
            const bool ok = active && e <= E && MBH_IN_RANGE(L.status, e, (long long)S.E_check + 1, kKernHetX, s);
            if (ok) {
                bool done = false;
                if (S.mix.xw[e].v[30] != 0.0f) {   // low-weight edge: float32 ratio
                    cf d32[3];
                    edge_delta_mixed_hm(wsd[lw], wsf[lw], wsh[lw], S.mix, e, S.modes, tob, d32);
                    if (f32_edge_small(d32)) {
                        f32_edge_df(d32, eta32[lw], dl);
                        done = true;
                    }
                }
                if (!done)
                    edge_delta_xhm(xw[lw], xh[lw], S.mix.xedge + e, S.mix.xgrp + (int64_t)e * 4, S.modes, tob, tab,
                                   dl);
            }
            c2f dp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dp[c].re.hi = __shfl_up_sync(0xffffffffu, dl[c].re.hi, 1, G);
                dp[c].re.lo = __shfl_up_sync(0xffffffffu, dl[c].re.lo, 1, G);
                dp[c].im.hi = __shfl_up_sync(0xffffffffu, dl[c].im.hi, 1, G);
                dp[c].im.lo = __shfl_up_sync(0xffffffffu, dl[c].im.lo, 1, G);
                if (lane == 0) dp[c] = carry[c];
                carry[c].re.hi = __shfl_sync(0xffffffffu, dl[c].re.hi, G - 1, G);
                carry[c].re.lo = __shfl_sync(0xffffffffu, dl[c].re.lo, G - 1, G);
                carry[c].im.hi = __shfl_sync(0xffffffffu, dl[c].im.hi, G - 1, G);
                carry[c].im.lo = __shfl_sync(0xffffffffu, dl[c].im.lo, G - 1, G);
            }
            if (ok) contract_x(S.mix.xw + e, dp, dl, adh, ahh);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const f2 odh = {__shfl_down_sync(0xffffffffu, adh.hi, o, G), __shfl_down_sync(0xffffffffu, adh.lo, o, G)};
            const f2 ohh = {__shfl_down_sync(0xffffffffu, ahh.hi, o, G), __shfl_down_sync(0xffffffffu, ahh.lo, o, G)};
            df_acc(adh, odh);
            df_acc(ahh, ohh);
        }
        if (lane == 0 && active) {
            const int64_t wi = w0 + lw;
            const double dh = S.mix.xsumA + df_to_double(adh);
            const double hh = S.mix.xsumB + df_to_double(ahh);
            L.out[wi] = -0.5 * (S.dd + hh - 2.0 * dh);
            L.out[L.W + wi] = dh;
            L.out[2 * L.W + wi] = hh;
        }
    }
}

// ------------------------------------------------------------------------------------------
// direct likelihood, fused, extended precision (MBH_MIXED, Sec. II Eqs. 2-3 over the full
// grid): every template point in double-float on the FP32 pipe (phase and time chain, orbit at
// t(f), amplitude, raw transfer), contracted in double-float with the data folded with the
// frequency-only factors K_c (xdirect_data_kernel)
// ------------------------------------------------------------------------------------------
constexpr int kDirXThreads = 256;

// Per-template constants: the float32 path's double-float phase and time chain (absolute), the
// response constants (absolute k/sqrt3, polarisation basis, mode factors) in an XWalker (its
// difference fields unused), the raw amplitude factor over sigma and 1/f_c^2.
struct XDirect {
    WalkerDF d;
    XWalker r;
    f2 amp, ifc2;
    float c1x;   // c1's third part: c1 ~ 2 pi t_ref reaches ~2e8, whose float pair is off by ~1e-6
    float c0x;   // c_0's third part and the relative residual of (pi M)^{-1/3}'s float pair:
    float icbr;  // Psi_PN ~ c_0 v^-5 reaches ~1e5 rad, where ~4e-15 of it is ~4e-10 rad
};

__device__ inline void xdirect_setup(const double* __restrict__ theta, int64_t W, int64_t i, double inv_sigma,
                                     XDirect& o)
{
    WalkerF wf;   // the float32 constants of the float32 path's set-up are not used here
    WalkerDFFull full;
    walker_setup_mixed(theta, W, i, o.d, wf, &full);
    // beyond the float pairs (both differences exact)
    o.c1x = (float)((full.c1 - (double)o.d.c1.hi) - (double)o.d.c1.lo);
    o.c0x = (float)((full.c0 - (double)o.d.c[0].hi) - (double)o.d.c[0].lo);
    o.icbr = (float)(((full.icb - (double)o.d.icbrt_piM.hi) - (double)o.d.icbrt_piM.lo) / full.icb);
    XDer x;
    xderive(theta, W, i, x);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        o.r.k3[j] = split_rn(x.k3[j]);
        o.r.ev[j] = split_rn(x.ev[j]);
    }
    o.r.eu[0] = split_rn(x.eu[0]);
    o.r.eu[1] = split_rn(x.eu[1]);
    o.r.Ga[0] = split_rn(x.G[0]);
    o.r.Ga[1] = split_rn(x.G[1]);
    o.r.Gb[0] = split_rn(x.G[2]);
    o.r.Gb[1] = split_rn(x.G[3]);
    // amp (pi M)^{-7/6}, the factor of the raw template (f^{-7/6} is folded into the data):
    // A = pi sqrt(2/3) M^2 sqrt(eta) / D v^{-7/2} exp(-(f/f_c)^2), v^{-7/2} = (pi M)^{-7/6} f^{-7/6}
    const double M = x.mt * kMsunSec;
    const double icb = rcbrt(kPi * M);
    const double amp76 = kPi * 0.816496580927726 * M * M * sqrt(x.eta) / x.dist * (icb * icb * icb) * sqrt(icb);
    o.amp = split_rn(amp76 * inv_sigma);
    o.ifc2 = split_rn(x.ifc2);
}

// Amplitude factor (2/m)^{-7/6} of the m-groups (order of hm_group_mask: m = 2, 3, 4, 1): a
// mode's v^{-7/2} at f2 = 2f/m is (pi M)^{-7/6} f^{-7/6} (2/m)^{-7/6}, and the folded data carry
// f^{-7/6}.
__constant__ f2 kGrpAmp[4] = {df_const(1.0), df_const(1.6048697909004944), df_const(2.2449240966187460),
                              df_const(0.44544935907016965)};

// One chain of the raw template H_c (h_c = K_c H_c) at one grid point, double-float: the (2,2)
// model at f2 = q2.f (the grid's f for the (2,2) mode; 2f/m for a higher-mode group), i.e. the
// phase and time chain at f2, the support test (f2 <= f_cut, t(f2) in [0, t_obs]), the orbit
// at t(f2), Phi = (m/2) Phi_22(f2), the amplitude (pi M)^{-7/6} exp(-(f2/f_c)^2)/sigma times
// ampr, and the raw transfer at the point's x of the mode factors times A e^{-i Phi}: the
// walker's (2,2) factors, or with kHM the group's modes' factors weighted by v^{p_lm}.
// q2: f2, f2^{1/3}, f2^{-1/3}, ln f2/3; fg the grid's f; x = pi f L/c with sin 2x, cos 2x.
// Phi = f c1 + f dk + (m/2) Psi_PN(f2) ((m/2) f2 = f): lin = f c1 mod 2 pi (x_direct_lin),
// the same for every mode.
template <bool kInl, bool kHM>
__device__ __forceinline__ bool x_direct_term(const XDirect& w, const XWalkerHM* wh, uint32_t gmask, const FreqDF& q2,
                                              f2 fg, f2 lin, float half_m, f2 ampr, f2 x, f2 s2, f2 c2, f2 tob,
                                              const SinTab& tab, c2f H[3])
{
    const WalkerDF& d = w.d;
    const f2 v = dd_mul_lazy(d.cbrt_piM, q2.f3);
    const f2 iv = dd_mul_lazy(d.icbrt_piM, q2.fm3);
    const f2 lnv = dd_add_lazy(d.ln_cbrt_piM, q2.lnf3);
    // Psi_PN = sum_k c_k v^{k-5} + ln v (cl5 + cl6 v) (c_1 = 0; the pinning constant in c_5), the
    // v^-k chain with its products' lo lo terms (dd_fma_full)
    f2 N = dd_mul_full(d.c[0], iv);
#pragma unroll
    for (int k = 2; k <= 5; ++k) N = dd_fma_full(N, iv, d.c[k]);
    const f2 Pp = dd_mul_lazy(dd_fma_lazy(d.c[7], v, d.c[6]), v);
    const f2 psi_pn = dd_add_lazy(dd_add_lazy(N, Pp), dd_mul_lazy(lnv, dd_fma_lazy(d.cl6, v, d.cl5)));
    // t(f2) = sum_k d_k v^{k-8} + dl6 v^{-2} ln v + t0 and the support test
    const f2 iv2 = dd_sqr_lazy(iv), iv4 = dd_sqr_lazy(iv2), iv8 = dd_sqr_lazy(iv4);
    f2 Q = d.d[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) Q = dd_fma_lazy(Q, v, d.d[k]);
    const f2 t = dd_add(dd_add_lazy(dd_mul_lazy(Q, iv8), dd_mul_lazy(dd_mul_lazy(lnv, d.dl6), iv2)), d.t0);
    if (!(dd_le(q2.f, d.fcut) && !dd_lt0(t) && dd_le(t, tob))) return false;
    // the residuals of c_0 and of (pi M)^{-1/3} beyond their float pairs, to first order: c0x v^-5
    // + icbr sum_k (5 - k) c_k v^{k-5}, k = 0..4 (float32; ~1e-8 rad at |Psi| ~ 1e6, the same
    // at every point: added once the phase is reduced, where it is not rounded away)
    float corr;
    {
        const float ivf = iv.hi;
        float dn = 5.0f * d.c[0].hi * ivf;
        dn = __fmaf_rn(dn, ivf, 3.0f * d.c[2].hi);
        dn = __fmaf_rn(dn, ivf, 2.0f * d.c[3].hi);
        dn = __fmaf_rn(dn, ivf, d.c[4].hi) * ivf;
        const float iv2f = ivf * ivf;
        corr = __fmaf_rn(w.c0x, iv2f * iv2f * ivf, w.icbr * dn);
    }
    // orbit angle at t: alpha(t_ref) + 2 pi (t - t_ref)/yr
    const SinCos oa = sincos_df<kInl>(dd_mul_lazy(dd_sub_lazy(t, d.tref), kOrbRate), tab);
    const f2 ds = dd_add_lazy(dd_mul_lazy(d.sa_ref, oa.cm1), dd_mul_lazy(d.ca_ref, oa.s));   // sin a - sin a_ref
    const f2 dc = dd_sub_lazy(dd_mul_lazy(d.ca_ref, oa.cm1), dd_mul_lazy(d.sa_ref, oa.s));   // cos a - cos a_ref
    const f2 sa = dd_add_lazy(d.sa_ref, ds), ca = dd_add_lazy(d.ca_ref, dc);
    // Phi_22(f2) = f2 (c1 + 2 pi AU/c k.(c(t) - c(t_ref))) + Psi_PN (c1 holds 2 pi t_ref -
    // psi'(f_max) and 2 pi AU/c k.c(t_ref); kx, ky carry 2 pi AU/c); a mode's phase is m/2 times
    // it (its Doppler term (m/2) f2 ... = f ...)
    const f2 dk = dd_add_lazy(dd_mul_lazy(d.kx, dc), dd_mul_lazy(d.ky, ds));
    const f2 pp = kHM && half_m != 1.0f ? dd_mul_f_lazy(psi_pn, half_m) : psi_pn;
    f2 phi = dd_add_lazy(dd_add_lazy(lin, dd_mul_lazy(fg, dk)), pp);
    if (fabsf(phi.hi) > 3.14f) phi = dd_reduce_2pi(phi);
    phi.lo = __fmaf_rn(kHM ? half_m : 1.0f, corr, phi.lo);
    const SinCos ph = sincos_df<kInl>(dd_norm(phi), tab);
    // raw amplitude amp (pi M)^{-7/6} exp(-(f2/f_c)^2)/sigma, Z = A e^{-i Phi} into the mode factors
    const f2 u = dd_mul_lazy(dd_sqr_lazy(q2.f), w.ifc2);
    f2 A = dd_mul_lazy(w.amp, dd_exp({-u.hi, -u.lo}));
    if (kHM) A = dd_mul_lazy(A, ampr);
    const c2f Z = {dd_add_lazy(A, dd_mul_lazy(A, ph.cm1)), dd_mul_lazy(A, {-ph.s.hi, -ph.s.lo})};
    f2 G[4] = {w.r.Ga[0], w.r.Ga[1], w.r.Gb[0], w.r.Gb[1]};
    if constexpr (kHM) {
        // the group's mode factors: sum of v^{p_lm} (Ga, Gb)_lm
#pragma unroll
        for (int j = 0; j < 4; ++j) G[j] = {0.0f, 0.0f};
        for (uint32_t bm = gmask; bm; bm &= bm - 1) {
            const int md = __ffs(bm) - 1;
            f2 vp = {1.0f, 0.0f};
            for (int j = 0; j < hm_vpow(md); ++j) vp = dd_mul_lazy(vp, v);
#pragma unroll
            for (int j = 0; j < 4; ++j) G[j] = dd_add_lazy(G[j], dd_mul_lazy(vp, wh->G[md][j]));
        }
    }
    const c2f za = cd_mul(Z, {G[0], G[1]}), zb = cd_mul(Z, {G[2], G[3]});
    const f2 zGa[2] = {za.re, za.im}, zGb[2] = {zb.re, zb.im};
    transfer_df<kInl>(w.r, zGa, zGb, x, s2, c2, sa, ca, tab, H);
    return true;
}

// f c1 modulo 2 pi with c1 as a triple-float (c1 ~ 2 pi t_ref reaches ~2e8, and f c1 ~1e7 rad)
__device__ __forceinline__ f2 x_direct_lin(const XDirect& w, f2 f) { return dd_mul_mod2pi(f, w.d.c1, w.c1x); }

// The raw template H_c of one template at one grid point, (2,2) mode (inlined bodies).
__device__ __forceinline__ bool point_x_direct(const XDirect& w, const FreqDF& q, f2 x, f2 s2, f2 c2, f2 tob,
                                               const SinTab& tab, c2f H[3])
{
    return x_direct_term<true, false>(w, nullptr, 0u, q, q.f, x_direct_lin(w, q.f), 1.0f, {1.0f, 0.0f}, x, s2, c2,
                                      tob, tab, H);
}

// The same summed over the modes of `modes` (Eq. 9): one chain and one transfer per distinct m
// (modes sharing m share f2, t(f2) and the orbit), the sine/cosine and arm bodies called out of
// line (the group loop's body would not fit the instruction cache inlined).  False when no
// mode is in its support.
__device__ __forceinline__ bool point_x_direct_hm(const XDirect& w, const XWalkerHM& wh, uint32_t modes,
                                                  const FreqDF& q, f2 x, f2 s2, f2 c2, f2 tob, const SinTab& tab,
                                                  c2f H[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) H[c] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    bool any = false;
    const f2 lin = x_direct_lin(w, q.f);
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
        const uint32_t gmask = modes & hm_group_mask(g);
        if (!gmask) continue;
        FreqDF q2 = q;
        if (g != 0)
            q2 = {dd_norm(dd_mul_lazy(q.f, kGrpR[g])), dd_norm(dd_mul_lazy(q.f3, kGrpR3[g])),
                  dd_norm(dd_mul_lazy(q.fm3, kGrpRm3[g])), dd_norm(dd_add_lazy(q.lnf3, kGrpLn3[g]))};
        c2f Hg[3];
        if (!x_direct_term<false, true>(w, &wh, gmask, q2, q.f, lin, kGrpHalfM[g], kGrpAmp[g], x, s2, c2, tob, tab, Hg))
            continue;
        any = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) H[c] = cd_add(H[c], Hg[c]);
    }
    return any;
}

// block (template tile of T, frequency chunk): the point's tables and folded data are loaded
// once and reused by the T templates; each thread keeps per-template double-float sums in
// shared memory, reduced per template at the end (float64) into part[template][chunk].  kHM:
// the templates of the modes of `modes` (point_x_direct_hm), else the (2,2) mode.
template <int T, bool kHM>
__global__ void __launch_bounds__(kDirXThreads)
    direct_fused_x_kernel(const double* __restrict__ theta, int64_t W, const float4* __restrict__ ft1,
                          const float4* __restrict__ ft2, const float4* __restrict__ ftx,
                          const float2* __restrict__ ftx2, double t_obs, const float4* __restrict__ wdx,
                          const float2* __restrict__ wvx, int64_t n, int64_t chunk, int nchunks, double inv_sigma,
                          uint32_t modes, double2* __restrict__ part)
{
    __shared__ XDirect ws[T];
    __shared__ XWalkerHM wsh[kHM ? T : 1];
    __shared__ SinTab tab;
    __shared__ float4 acc[T][kDirXThreads];   // per template: <d|h> hi, lo, <h|h> hi, lo
    __shared__ double sm[32 * 2];
    __shared__ f2 s_tob;
    const int64_t w0 = (int64_t)blockIdx.x * T;
    const int ch = blockIdx.y;
    const int nt = (int)std::min<int64_t>(T, W - w0);
    load_sintab(tab);
    if (threadIdx.x < nt) xdirect_setup(theta, W, w0 + threadIdx.x, inv_sigma, ws[threadIdx.x]);
    if (kHM && threadIdx.x >= 32 && threadIdx.x < 32 + nt)   // on another warp
        xwalker_setup_hm(theta, W, w0 + threadIdx.x - 32, wsh[threadIdx.x - 32]);
    if (threadIdx.x == 0) s_tob = split_rn(t_obs);
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t][threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const f2 tob = s_tob;
    const int64_t kb = (int64_t)ch * chunk, ke = std::min<int64_t>(n, kb + chunk);
    for (int64_t k = kb + threadIdx.x; k < ke; k += kDirXThreads) {
        const float4 a = __ldg(ft1 + k), b = __ldg(ft2 + k), xa = __ldg(ftx + k);
        const float2 xb = __ldg(ftx2 + k);
        const FreqDF q = {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}, {b.z, b.w}};
        const f2 x = {xa.x, xa.y}, s2 = {xa.z, xa.w}, c2 = {xb.x, xb.y};
        c2f D[3];
        f2 V[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 dv = __ldg(wdx + (int64_t)c * n + k);
            const float2 vv = __ldg(wvx + (int64_t)c * n + k);
            D[c] = {{dv.x, dv.y}, {dv.z, dv.w}};
            V[c] = {vv.x, vv.y};
        }
        for (int t = 0; t < nt; ++t) {
            c2f H[3];
            if (kHM ? !point_x_direct_hm(ws[t], wsh[t], modes, q, x, s2, c2, tob, tab, H)
                    : !point_x_direct(ws[t], q, x, s2, c2, tob, tab, H))
                continue;
            f2 sd = {0.0f, 0.0f}, sh = {0.0f, 0.0f};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // Re conj(conj(K) D) H = Re conj(D) h; |H|^2 |K|^2 V = |h|^2 V.  The squares keep
                // lo^2: after the transfer's cancellations H's parts can be unnormalised (|lo|
                // well above ulp(hi)), and a dropped lo^2 (never negative) biases <h|h> low
                sd = dd_add_lazy(sd, dd_add_lazy(dd_mul_lazy(D[c].re, H[c].re), dd_mul_lazy(D[c].im, H[c].im)));
                sh = dd_add_lazy(sh, dd_mul_lazy(V[c], dd_add_lazy(dd_sqr_full(H[c].re), dd_sqr_full(H[c].im))));
            }
            float4 s = acc[t][threadIdx.x];
            f2 adh = {s.x, s.y}, ahh = {s.z, s.w};
            df_acc(adh, sd);
            df_acc(ahh, sh);
            acc[t][threadIdx.x] = make_float4(adh.hi, adh.lo, ahh.hi, ahh.lo);
        }
    }
    for (int t = 0; t < nt; ++t) {
        const float4 s = acc[t][threadIdx.x];
        double r[2] = {df_to_double({s.x, s.y}), df_to_double({s.z, s.w})};
        block_sum<2>(r, sm);
        if (threadIdx.x == 0) part[(w0 + t) * nchunks + ch] = make_double2(r[0], r[1]);
    }
}

// The extended direct pass's tables of one data set: per grid point x = pi f L/c with sin 2x,
// cos 2x, and per channel the data with the frequency-only factors folded in (float64, split
// once): conj(K_c) sigma 4 df d/S and |K_c|^2 sigma^2 4 df/S, with K_c the factors that the raw
// transfer leaves out (including f^{-7/6}, as the float32 pass's folded data).
__global__ void xdirect_data_kernel(double f0, double df, int64_t n, double sigma, const double2* __restrict__ wd,
                                    const double* __restrict__ wv, float4* __restrict__ ftx,
                                    float2* __restrict__ ftx2, float4* __restrict__ wdx, float2* __restrict__ wvx)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double f = f0 + (double)k * df;
        const double x = kPi * kArmSec * f;
        double s1, c1, s2x, c2x, s3, c3;
        sincos(x, &s1, &c1);
        sincos(2.0 * x, &s2x, &c2x);
        sincos(3.0 * x, &s3, &c3);
        const f2 xs = split_rn(x), ss = split_rn(s2x), cs = split_rn(c2x);
        ftx[k] = make_float4(xs.hi, xs.lo, ss.hi, ss.lo);
        ftx2[k] = make_float2(cs.hi, cs.lo);
        // K: W = (1 - D^2)(-x) e^{-ix} f^{-7/6}, 1 - D = 2 sin x (sin x, cos x), D = e^{-2ix};
        // K_A = W/sqrt2, K_E = W/sqrt6, K_T = W (1 - D)/sqrt3
        const double wm = -2.0 * x * s2x * pow(f, -7.0 / 6.0);
        const double wr = wm * s3, wi = wm * c3;
        const double ar = 2.0 * s1 * s1, ai = 2.0 * s1 * c1;
        const double Kr[3] = {wr / kSqrt2, wr / kSqrt6, (wr * ar - wi * ai) / kSqrt3};
        const double Ki[3] = {wi / kSqrt2, wi / kSqrt6, (wr * ai + wi * ar) / kSqrt3};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 d = wd[c * n + k];
            const double dr = sigma * d.x, di = sigma * d.y;
            const f2 re = split_rn(Kr[c] * dr + Ki[c] * di), im = split_rn(Kr[c] * di - Ki[c] * dr);
            wdx[c * n + k] = make_float4(re.hi, re.lo, im.hi, im.lo);
            const f2 vv = split_rn(sigma * sigma * wv[c * n + k] * (Kr[c] * Kr[c] + Ki[c] * Ki[c]));
            wvx[c * n + k] = make_float2(vv.hi, vv.lo);
        }
    }
}

// ------------------------------------------------------------------------------------------
// reference tables
// ------------------------------------------------------------------------------------------
__global__ void xref_kernel(const double* __restrict__ theta0, XDer* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) xderive(theta0, 1, 0, *out);
}

// Edge records: the reference's v0, 1/v0, ln v0, t0(f), its orbit angle alpha0 = 2 pi t0/yr, the
// one-link phase x = pi f L/c with sin 2x, cos 2x, and G_c = K_c/T0_c (float64: T0_c the
// reference's full transfer at alpha0, K_c the frequency-only factors that the raw transfer
// leaves out), 0 where h0 = 0.
__global__ void xedge_kernel(const double* __restrict__ theta0, const XDer* __restrict__ xr, double t_obs,
                             const double* __restrict__ fe, int n_edges, XEdge* __restrict__ out)
{
    __shared__ Walker w;
    if (threadIdx.x == 0) walker_setup(theta0, 1, 0, w, 1u);
    __syncthreads();
    const XDer& r = *xr;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += gridDim.x * blockDim.x) {
        const double f = fe[e];
        const double v0 = cbrt(kPi * r.mt * kMsunSec * f), iv0 = 1.0 / v0, lnv0 = log(v0);
        double Q = r.d[7];
        for (int k = 6; k >= 0; --k) Q = fma(Q, v0, r.d[k]);
        const double iv2 = iv0 * iv0, iv8 = iv2 * iv2 * iv2 * iv2;
        const double t0 = Q * iv8 + r.dl6 * lnv0 * iv2 + r.t0;
        double sa0, ca0;
        sincos(kTwoPi * t0 / kYear, &sa0, &ca0);
        const double x = kPi * kArmSec * f;
        double s1, c1, s2x, c2x, s3, c3;
        sincos(x, &s1, &c1);
        sincos(2.0 * x, &s2x, &c2x);
        sincos(3.0 * x, &s3, &c3);
        XEdge m;
        const f2 vals[10] = {split_rn(f), split_rn(v0), split_rn(iv0), split_rn(lnv0), split_rn(t0),
                             split_rn(ca0), split_rn(sa0), split_rn(x), split_rn(s2x), split_rn(c2x)};
        float* p = reinterpret_cast<float*>(&m);
        for (int j = 0; j < 10; ++j) {
            p[2 * j] = vals[j].hi;
            p[2 * j + 1] = vals[j].lo;
        }
        // the reference's support (as its float64 template): h0 = 0 outside
        cd h0[3];
        const bool in = point_f64(w, f, t_obs, h0);
        cd T0[3];
        transfer_f64(w, f, sa0, ca0, w.Kp, w.Kc, T0);
        // K: W = (1 - D^2)(-x) e^{-ix} = -2 x sin2x (sin3x, cos3x), 1 - D = 2 sin x (sin x, cos x);
        // K_A = W/sqrt2, K_E = W/sqrt6, K_T = W (1 - D)/sqrt3
        const double wm = -2.0 * x * s2x;
        const double wr = wm * s3, wi = wm * c3;
        const double ar = 2.0 * s1 * s1, ai = 2.0 * s1 * c1;
        const cd K[3] = {{wr / kSqrt2, wi / kSqrt2}, {wr / kSqrt6, wi / kSqrt6},
                         {(wr * ar - wi * ai) / kSqrt3, (wr * ai + wi * ar) / kSqrt3}};
        for (int c = 0; c < 3; ++c) {
            const double m2 = T0[c].re * T0[c].re + T0[c].im * T0[c].im;
            double gr = 0.0, gi = 0.0;
            if (in && m2 > 0.0 && (h0[c].re != 0.0 || h0[c].im != 0.0)) {
                gr = (K[c].re * T0[c].re + K[c].im * T0[c].im) / m2;
                gi = (K[c].im * T0[c].re - K[c].re * T0[c].im) / m2;
            }
            const f2 a = split_rn(gr), b = split_rn(gi);
            p[20 + 4 * c] = a.hi;
            p[21 + 4 * c] = a.lo;
            p[22 + 4 * c] = b.hi;
            p[23 + 4 * c] = b.lo;
        }
        out[e] = m;
    }
}

// Higher-mode reference: the edge records' shared part (f, v0, 1/v0, ln v0 at f, x, sin 2x,
// cos 2x; the (2,2) slots t0, cos/sin alpha0 and G of group m = 2 are also filled) and per mode
// group g (m = 2, 3, 4, 1) the group's t0(f2), orbit angle at it and
//   G_gc = A0(f2) e^{-i Phi0_g(f)} K_c / h0_c,
// float64: A0(f2) the reference's (2,2) amplitude at f2 = 2f/m, Phi0_g the group's large phase
// ((m/2) times the (2,2) phase at f2, plus 2 pi f k0.c(t0(f2))), K_c the frequency-only factors
// of the raw transfer and h0 the sum of the reference's modes; 0 where h0 = 0.
__global__ void xedge_hm_kernel(const double* __restrict__ theta0, uint32_t modes, const XDer* __restrict__ xr,
                                double t_obs, const double* __restrict__ fe, int n_edges, XEdge* __restrict__ out,
                                XGrp* __restrict__ grp)
{
    __shared__ Walker w;
    if (threadIdx.x == 0) walker_setup(theta0, 1, 0, w, modes);
    __syncthreads();
    const XDer& r = *xr;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_edges; e += gridDim.x * blockDim.x) {
        const double f = fe[e];
        const double x = kPi * kArmSec * f;
        double s1, c1, s2x, c2x, s3, c3;
        sincos(x, &s1, &c1);
        sincos(2.0 * x, &s2x, &c2x);
        sincos(3.0 * x, &s3, &c3);
        const double wm = -2.0 * x * s2x;
        const double wr = wm * s3, wi = wm * c3;
        const double ar = 2.0 * s1 * s1, ai = 2.0 * s1 * c1;
        const cd K[3] = {{wr / kSqrt2, wi / kSqrt2}, {wr / kSqrt6, wi / kSqrt6},
                         {(wr * ar - wi * ai) / kSqrt3, (wr * ai + wi * ar) / kSqrt3}};
        cd h0[3];
        point_hm_f64(w, f, t_obs, h0);
        XEdge m;
        float* p = reinterpret_cast<float*>(&m);
        for (int j = 0; j < 32; ++j) p[j] = 0.0f;
        for (int g = 0; g < 4; ++g) {
            float* q = reinterpret_cast<float*>(grp + (int64_t)e * 4 + g);
            for (int j = 0; j < 20; ++j) q[j] = 0.0f;
            const int mm = g == 0 ? 2 : g == 1 ? 3 : g == 2 ? 4 : 1;
            const double f2v = 2.0 * f / mm;
            const double v0 = cbrt(kPi * r.mt * kMsunSec * f2v), iv0 = 1.0 / v0, lnv0 = log(v0);
            double Q = r.d[7];
            for (int k = 6; k >= 0; --k) Q = fma(Q, v0, r.d[k]);
            const double iv2 = iv0 * iv0, iv8 = iv2 * iv2 * iv2 * iv2;
            const double t0 = Q * iv8 + r.dl6 * lnv0 * iv2 + r.t0;
            double sa0, ca0;
            sincos(kTwoPi * t0 / kYear, &sa0, &ca0);
            if (g == 0) {   // shared part (at f: group m = 2)
                const f2 vals[10] = {split_rn(f), split_rn(v0), split_rn(iv0), split_rn(lnv0), split_rn(t0),
                                     split_rn(ca0), split_rn(sa0), split_rn(x), split_rn(s2x), split_rn(c2x)};
                for (int j = 0; j < 10; ++j) {
                    p[2 * j] = vals[j].hi;
                    p[2 * j + 1] = vals[j].lo;
                }
            }
            if (!(modes & hm_group_mask(g))) continue;
            const f2 tv[3] = {split_rn(t0), split_rn(ca0), split_rn(sa0)};
            for (int j = 0; j < 3; ++j) {
                q[2 * j] = tv[j].hi;
                q[2 * j + 1] = tv[j].lo;
            }
            // the reference's (2,2) amplitude at f2 and the group's phase, float64
            const double vw = cbrt(w.piM * f2v);
            double psi_pn, dpsi_pn;
            pn_phase_f64(w, vw, log(vw), psi_pn, dpsi_pn);
            const double tg = w.tref + (dpsi_pn - w.dpsi_max) * kInvTwoPi;
            double sa, ca;
            sincos(kTwoPi * tg / kYear, &sa, &ca);
            const double kc = kAUSec * (w.k[0] * ca + w.k[1] * sa);
            const double Phi = 0.5 * mm * (kTwoPi * f2v * w.tref + psi_pn - w.psi_max - (f2v - w.fmax) * w.dpsi_max) +
                               kTwoPi * f * kc;
            const double amp = w.amp * exp(-f2v * f2v * w.inv_fc2) / (vw * vw * vw * sqrt(vw));
            double sP, cP;
            sincos(Phi, &sP, &cP);
            for (int c = 0; c < 3; ++c) {
                const double m2 = h0[c].re * h0[c].re + h0[c].im * h0[c].im;
                double gr = 0.0, gi = 0.0;
                if (m2 > 0.0) {
                    // amp e^{-i Phi} K_c / h0_c
                    const double nr = amp * (cP * K[c].re + sP * K[c].im), ni = amp * (cP * K[c].im - sP * K[c].re);
                    gr = (nr * h0[c].re + ni * h0[c].im) / m2;
                    gi = (ni * h0[c].re - nr * h0[c].im) / m2;
                }
                const f2 a = split_rn(gr), b = split_rn(gi);
                q[8 + 4 * c] = a.hi;
                q[9 + 4 * c] = a.lo;
                q[10 + 4 * c] = b.hi;
                q[11 + 4 * c] = b.lo;
            }
        }
        out[e] = m;
    }
}

// Per-edge contraction weights (factor 4 included) from the summary data of the edge's two bins
// (bin e as its lower edge, bin e - 1 as its upper edge), and the constant parts 4 sum Re A0,
// 4 sum B0.
__global__ void xweight_kernel(const double* __restrict__ summary, const double* __restrict__ invw, int E,
                               XWeight* __restrict__ out, double* __restrict__ sums, double* __restrict__ sens)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e <= E) {
        XWeight m;
        float* p = reinterpret_cast<float*>(&m);
        for (int j = 0; j < 32; ++j) p[j] = 0.0f;
        double S = 0.0;
        for (int c = 0; c < 3; ++c) {
            double war = 0.0, wai = 0.0, wbr = 0.0, wq = 0.0, wc = 0.0;
            if (e < E) {   // lower edge of bin e
                const double* q = summary + ((int64_t)e * 3 + c) * 6;
                const double iw = invw[e];
                war += 0.5 * q[0] - q[2] * iw;
                wai += 0.5 * q[1] - q[3] * iw;
                wbr += q[4] - 2.0 * q[5] * iw;
                wq += 0.25 * q[4] - q[5] * iw;
            }
            if (e >= 1) {   // upper edge of bin e - 1
                const double* q = summary + ((int64_t)(e - 1) * 3 + c) * 6;
                const double iw = invw[e - 1];
                war += 0.5 * q[0] + q[2] * iw;
                wai += 0.5 * q[1] + q[3] * iw;
                wbr += q[4] + 2.0 * q[5] * iw;
                wq += 0.25 * q[4] + q[5] * iw;
                wc = 0.5 * q[4];
            }
            const f2 v[4] = {split_rn(4.0 * war), split_rn(4.0 * wai), split_rn(4.0 * wbr), split_rn(4.0 * wq)};
            for (int j = 0; j < 4; ++j) {
                p[8 * c + 2 * j] = v[j].hi;
                p[8 * c + 2 * j + 1] = v[j].lo;
            }
            const f2 cc = split_rn(4.0 * wc);
            p[24 + 2 * c] = cc.hi;
            p[25 + 2 * c] = cc.lo;
            // |d lnL / d delta| bound for |delta| and its neighbours' <= kDeltaMax (lnL = <d|h> -
            // <h|h>/2 + const): the linear weights, 2 kDeltaMax |wq|, kDeltaMax |wc| (the cross
            // term with the previous edge) and kDeltaMax |wcn|, the next edge's cross term with
            // this one (its wc: 0.5 B0 of bin e)
            const double wcn = e < E ? 0.5 * summary[((int64_t)e * 3 + c) * 6 + 4] : 0.0;
            S += 4.0 * (fabs(war) + fabs(wai) + 0.5 * fabs(wbr) + kDeltaMax * fabs(wq) +
                        0.5 * kDeltaMax * (fabs(wc) + fabs(wcn)));
        }
        out[e] = m;
        sens[e] = S;
    }
    if (e == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < E; ++i)
            for (int c = 0; c < 3; ++c) {
                a += summary[((int64_t)i * 3 + c) * 6 + 0];
                b += summary[((int64_t)i * 3 + c) * 6 + 4];
            }
        sums[0] = 4.0 * a;
        sums[1] = 4.0 * b;
    }
}

// The edges that take the float32 ratio: the least sensitive groups of kF32Group aligned edges
// (a group's sensitivity: the sum of its S_e (xweight_kernel) times kappa_e, 1 without higher
// modes), in ascending order while kF32EdgeError x (sum of their sensitivities) stays within
// kF32Budget; flagged in v[30] of their weight records.  Reads back the constant parts and sets
// R->mix's extended-precision fields.
static cudaError_t select_f32_edges(mbh_ref* R, cudaStream_t st, const std::vector<double>* kappa)
{
    const int E = R->E;
    double sums[2];
    std::vector<double> sens(E + 1);
    cudaError_t e = cudaMemcpyAsync(sums, R->x_sums, sizeof sums, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sens.data(), R->x_sens, sizeof(double) * (E + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const int ng = (E + 1 + kF32Group - 1) / kF32Group;
    std::vector<double> gs(ng, 0.0);
    for (int i = 0; i <= E; ++i) gs[i / kF32Group] += sens[i] * (kappa ? (*kappa)[i] : 1.0);
    std::vector<int> order(ng);
    for (int i = 0; i < ng; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gs[a] < gs[b]; });
    std::vector<float> flag(E + 1, 0.0f);
    double acc = 0.0;
    int n32 = 0;
    for (int gi : order) {
        if (kF32EdgeError * (acc + gs[gi]) > kF32Budget) break;
        acc += gs[gi];
        for (int i = gi * kF32Group; i < std::min(E + 1, (gi + 1) * kF32Group); ++i) {
            flag[i] = 1.0f;
            ++n32;
        }
    }
    // v[30] of every record (pitch sizeof(XWeight))
    e = cudaMemcpy2DAsync(reinterpret_cast<char*>(R->x_w) + 30 * sizeof(float), sizeof(XWeight), flag.data(),
                          sizeof(float), sizeof(float), E + 1, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        R->mix.xder = R->x_der;
        R->mix.xedge = R->x_edge;
        R->mix.xw = R->x_w;
        R->mix.xsumA = sums[0];
        R->mix.xsumB = sums[1];
        R->mix.xn32 = n32;
    }
    return e;
}

// Tables of the extended-precision heterodyne for a (2,2) reference: XDer of theta0, edge
// records, edge weights and the constant parts, and the float32-ratio edges (select_f32_edges).
cudaError_t prepare_x_tables(mbh_ref* R, cudaStream_t st)
{
    const int E = R->E;
    cudaError_t e = cudaMalloc(&R->x_der, sizeof(XDer));
    if (e == cudaSuccess) e = cudaMalloc(&R->x_edge, sizeof(XEdge) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->x_w, sizeof(XWeight) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->x_sums, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&R->x_sens, sizeof(double) * (E + 1));
    if (e != cudaSuccess) return e;
    xref_kernel<<<1, 32, 0, st>>>(R->theta0_dev, R->x_der);
    xedge_kernel<<<(E + 1 + 127) / 128, 128, 0, st>>>(R->theta0_dev, R->x_der, R->grid.t_obs, R->fe, E + 1,
                                                      R->x_edge);
    xweight_kernel<<<(E + 1 + 127) / 128, 128, 0, st>>>(R->summary, R->invw, E, R->x_w, R->x_sums, R->x_sens);
    e = cudaGetLastError();
    return e == cudaSuccess ? select_f32_edges(R, st, nullptr) : e;
}

// Tables of the extended-precision heterodyne for a higher-mode reference: XDer of theta0, the
// edge records and the per-group records, the edge weights and the constant parts, and the
// float32-ratio edges (select_f32_edges; their ratio from the float32 higher-mode tables).
cudaError_t prepare_x_tables_hm(mbh_ref* R, cudaStream_t st)
{
    const int E = R->E;
    cudaError_t e = cudaMalloc(&R->x_der, sizeof(XDer));
    if (e == cudaSuccess) e = cudaMalloc(&R->x_edge, sizeof(XEdge) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->x_grp, sizeof(XGrp) * 4 * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->x_w, sizeof(XWeight) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&R->x_sums, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&R->x_sens, sizeof(double) * (E + 1));
    if (e != cudaSuccess) return e;
    xref_kernel<<<1, 32, 0, st>>>(R->theta0_dev, R->x_der);
    xedge_hm_kernel<<<(E + 1 + 127) / 128, 128, 0, st>>>(R->theta0_dev, R->modes, R->x_der, R->grid.t_obs, R->fe,
                                                         E + 1, R->x_edge, R->x_grp);
    xweight_kernel<<<(E + 1 + 127) / 128, 128, 0, st>>>(R->summary, R->invw, E, R->x_w, R->x_sums, R->x_sens);
    e = cudaGetLastError();
    // kappa_e = max over channels of sum over mode groups |u_g| (the float32 higher-mode records)
    std::vector<MixModeHM> hm((size_t)(E + 1) * kHmModes);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hm.data(), R->mix_hm, sizeof(MixModeHM) * hm.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::vector<double> kappa(E + 1, 1.0);
    for (int i = 0; i <= E; ++i) {
        double kmax = 1.0;
        for (int c = 0; c < 3; ++c) {
            double k = 0.0;
            for (int g = 0; g < 4; ++g) {
                const uint32_t gmask = R->modes & hm_group_mask(g);
                if (!gmask) continue;
                const float2 u = hm[(size_t)i * kHmModes + (__builtin_ctz(gmask))].u[c];
                k += std::hypot((double)u.x, (double)u.y);
            }
            kmax = std::max(kmax, k);
        }
        kappa[i] = kmax;
    }
    e = select_f32_edges(R, st, &kappa);
    if (e == cudaSuccess) R->mix.xgrp = R->x_grp;
    return e;
}

mbh_status make_x_direct_tables(mbh_data* D, cudaStream_t st)
{
    const int64_t n = D->grid.n;
    cudaError_t e = cudaMalloc(&D->ftx, sizeof(float4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->ftx2, sizeof(float2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->wdx, sizeof(float4) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&D->wvx, sizeof(float2) * 3 * n);
    if (e != cudaSuccess) return cuda_fail(e, "extended direct tables");
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32);
    xdirect_data_kernel<<<blocks, 256, 0, st>>>(D->grid.f0, D->grid.df, n, D->sigma, D->wd, D->wv, D->ftx, D->ftx2,
                                                 D->wdx, D->wvx);
    e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "extended direct tables");
}

mbh_status launch_direct_fused_x(const mbh_data* data, const double* theta, int64_t W, double* out,
                                 cudaStream_t st, uint32_t modes)
{
    constexpr int T = 4;
    const int64_t tiles = (W + T - 1) / T;
    if (tiles > 0x7fffffff) return fail(MBH_EINVAL, "W too large");
    int64_t chunk;
    int nchunks;
    // one wave of blocks (2 per SM) at least: each block's float64 set-up of its 4 templates is
    // worth ~1000 points of their double-float work
    direct_chunks(data->grid.n, tiles, 1 << 14, chunk, nchunks, 2);
    double2* part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, sizeof(double2) * W * nchunks, st);
    if (e != cudaSuccess) return cuda_fail(e, "direct_loglike_batch alloc");
    dim3 grid((unsigned)tiles, (unsigned)nchunks);
    if (modes == 1u)
        direct_fused_x_kernel<T, false><<<grid, kDirXThreads, 0, st>>>(
            theta, W, data->ftab, data->ftab2, data->ftx, data->ftx2, data->grid.t_obs, data->wdx, data->wvx,
            data->grid.n, chunk, nchunks, 1.0 / data->sigma, modes, part);
    else
        direct_fused_x_kernel<T, true><<<grid, kDirXThreads, 0, st>>>(
            theta, W, data->ftab, data->ftab2, data->ftx, data->ftx2, data->grid.t_obs, data->wdx, data->wvx,
            data->grid.n, chunk, nchunks, 1.0 / data->sigma, modes, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(part, st);
        return cuda_fail(e, "direct_fused_x_kernel");
    }
    return direct_finish(part, nchunks, W, data->dd, out, st);
}

// Test support (mbh_selftest_math kinds 5 and 6): the double-float sine/cosine of (x[2i],
// x[2i+1]) as given (normalised or not) into o1 (sin) and o2 (cos - 1) as (hi, lo) pairs; the
// exactly reduced product (x[2i], x[2i+1]) (y[3i], y[3i+1], y[3i+2]) mod 2 pi into o1.
__global__ void selftest_df_kernel(int kind, const float* __restrict__ x, const float* __restrict__ y, int64_t n,
                                   float* __restrict__ o1, float* __restrict__ o2)
{
    __shared__ SinTab tab;
    load_sintab(tab);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const f2 a = {x[2 * i], x[2 * i + 1]};
        if (kind == 5) {
            f2 sn, cm;
            dd_sincos_any(a, tab, sn, cm);
            o1[2 * i] = sn.hi;
            o1[2 * i + 1] = sn.lo;
            o2[2 * i] = cm.hi;
            o2[2 * i + 1] = cm.lo;
        } else {
            const f2 r = dd_mul_mod2pi(a, {y[3 * i], y[3 * i + 1]}, y[3 * i + 2]);
            o1[2 * i] = r.hi;
            o1[2 * i + 1] = r.lo;
        }
    }
}

mbh_status selftest_df(int kind, const float* x, const float* y, int64_t n, float* o1, float* o2, cudaStream_t st)
{
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 32);
    selftest_df_kernel<<<blocks, 256, 0, st>>>(kind, x, y, n, o1, o2);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "mbh_selftest_math");
}

void free_x_tables(mbh_ref* R)
{
    if (R->x_der) cudaFree(R->x_der);
    if (R->x_edge) cudaFree(R->x_edge);
    if (R->x_w) cudaFree(R->x_w);
    if (R->x_sums) cudaFree(R->x_sums);
    if (R->x_sens) cudaFree(R->x_sens);
    if (R->x_grp) cudaFree(R->x_grp);
}

}  // namespace mbh

namespace {
template <int G, int BLOCK>
cudaError_t launch_het_x(const HetLaunch& L, int grid, cudaStream_t st)
{
    het_x_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}

template <int G, int BLOCK>
cudaError_t launch_het_x_pt(const HetLaunch& L, int grid, cudaStream_t st)
{
    het_x_pt_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}

template <int G, int BLOCK>
cudaError_t launch_het_xhm(const HetLaunch& L, int grid, cudaStream_t st)
{
    het_xhm_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}
}  // namespace

namespace mbh {
HetKernel het_kernel_x(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return {&launch_het_x<g, b>, (const void*)&het_x_kernel<g, b>};
    MBH_CASE(1, 64) MBH_CASE(1, 128) MBH_CASE(1, 256)
    MBH_CASE(2, 64) MBH_CASE(2, 128) MBH_CASE(2, 256)
    MBH_CASE(4, 64) MBH_CASE(4, 128) MBH_CASE(4, 256) MBH_CASE(4, 96) MBH_CASE(4, 160) MBH_CASE(4, 224)
    MBH_CASE(8, 64) MBH_CASE(8, 128) MBH_CASE(8, 256)
    MBH_CASE(16, 64) MBH_CASE(16, 128) MBH_CASE(16, 256)
    MBH_CASE(32, 64) MBH_CASE(32, 128) MBH_CASE(32, 256)
#undef MBH_CASE
    return {nullptr, nullptr};
}
}  // namespace mbh

namespace mbh {
// fused sampler half steps of the extended kernel: blocks of at most 32 walkers
HetKernel het_kernel_x_pt(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return {&launch_het_x_pt<g, b>, (const void*)&het_x_pt_kernel<g, b>};
    MBH_CASE(2, 64) MBH_CASE(4, 64) MBH_CASE(4, 128) MBH_CASE(8, 128) MBH_CASE(8, 256)
    MBH_CASE(16, 256) MBH_CASE(32, 256)
#undef MBH_CASE
    return {nullptr, nullptr};
}

HetKernel het_kernel_xhm(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return {&launch_het_xhm<g, b>, (const void*)&het_xhm_kernel<g, b>};
    MBH_CASE(1, 64) MBH_CASE(1, 128)
    MBH_CASE(2, 64) MBH_CASE(2, 128) MBH_CASE(2, 256)
    MBH_CASE(4, 64) MBH_CASE(4, 128) MBH_CASE(4, 256)
    MBH_CASE(8, 64) MBH_CASE(8, 128) MBH_CASE(8, 256)
    MBH_CASE(16, 64) MBH_CASE(16, 128) MBH_CASE(16, 256)
    MBH_CASE(32, 64) MBH_CASE(32, 128) MBH_CASE(32, 256)
#undef MBH_CASE
    return {nullptr, nullptr};
}
}  // namespace mbh

// Device model of the batched LISA MBHB likelihood (Katz, arXiv:2111.01064, Sec. II A):
// per-walker constants (parameter derivation), the "W0" amplitude/phase of the (2,2) mode
// (Eq. 7) with t(f) from the SPA (Eq. 8), and the "R0" A/E/T response (Eqs. 4-6, 9).
//
// Template at frequency f:
//   h~_c(f) = A(f) e^{-i Phi(f)} T_c(f),   Phi = Psi + 2 pi f k.c(t(f)),
// where Psi is the W0 phase, c(t) the constellation's guiding centre (seconds), and T_c
// the transfer of channel c with only O(1) phases left in it (the arm phases measured from
// the guiding centre, the sinc factors, the TDI delays and the mode/polarisation factors).
// Keeping the large phase Phi separate is what lets the mixed-precision path keep just Phi
// and t(f) in float64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mbh {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kInvTwoPi = 0.159154943091895335768883763372514362;
constexpr double kMsunSec = 4.925490947641267e-6;   // G Msun / c^3
constexpr double kClight = 299792458.0;
constexpr double kParsec = 3.085677581491367e16;
constexpr double kAU = 1.495978707e11;
constexpr double kYear = 31557600.0;                 // Julian year
constexpr double kArm = 2.5e9;                       // LISA arm length (m)
constexpr double kArmSec = kArm / kClight;
constexpr double kAUSec = kAU / kClight;
constexpr double kEulerGamma = 0.5772156649015328606;
constexpr double kSqrt3 = 1.732050807568877293527446341505872367;
constexpr double kSqrt2 = 1.414213562373095048801688724209698079;
constexpr double kSqrt6 = 2.449489742783178098197284074705891392;

enum { kMT = 0, kQ, kA1, kA2, kDL, kPhi, kIota, kLam, kBeta, kPsi, kTref, kNParams };

// Per-walker constants, computed once per walker by one thread.
struct Walker {
    double piM;             // pi * M_total (s)
    double cbrt_piM;        // (pi M)^{1/3}
    double icbrt_piM;       // (pi M)^{-1/3}
    double ln_cbrt_piM;     // ln((pi M)^{1/3})
    double tref, fmax, fcut, inv_fc2;
    double amp;             // A = amp v^{-7/2} exp(-f^2 inv_fc2) inside the support
    double c[8];            // Psi_PN = v^{-5} (sum_k c_k v^k + ln v (cl5 v^5 + cl6 v^6))
    double cl5, cl6;
    double d[8];            // dPsi_PN/df = v^{-8} (sum_k d_k v^k + dl6 v^6 ln v)
    double dl6;
    double psi_max, dpsi_max;
    double sa_ref, ca_ref;  // sin, cos of the orbital angle at t_ref
    double k[3];            // propagation direction
    double Pp[6], Pc[6];    // polarisation tensors (xx, xy, xz, yy, yz, zz)
    double Kp[2], Kc[2];    // mode factors of h+ and hx (complex)
    uint32_t modes;         // bit b: mode (kHmL[b], kHmM[b]); 1 = the (2,2) mode alone (W0)
    double hk[6][4];        // per mode: K+ and Kx (re, im) times H_lm's constant and sqrt(2/m)
};

// Higher harmonics ("W0-HM", Sec. II A, Eqs. 7-9): mode (l, m) uses the (2,2) phase at
// f2 = 2f/m scaled by m/2, so t_lm(f) = t_22(f2) (Eq. 8), the (2,2) amplitude at f2 times
// sqrt(2/m) (stationary phase for harmonic m of the same orbital phase) times the leading
// post-Newtonian mode factor H_lm = c_lm x^{p_lm} (Blanchet, Faye, Iyer & Sinha 2008),
// x = v^2 with v = (pi M f2)^{1/3}; each mode has its own response at t_lm (Eq. 9).
constexpr int kHmModes = 6;
__host__ __device__ constexpr int hm_m(int b) { return b == 0 ? 2 : b == 1 ? 3 : b == 2 ? 4 : b == 3 ? 1 : b == 4 ? 2 : 3; }
__host__ __device__ constexpr int hm_vpow(int b) { return b == 0 ? 0 : b == 1 ? 1 : b == 2 ? 2 : b == 3 ? 1 : b == 4 ? 2 : 3; }
constexpr uint32_t kHmAll = 0x3Fu;

// TaylorF2-type phase and its frequency derivative from v and ln v (Horner form).
__device__ __forceinline__ void pn_phase_f64(const Walker& w, double v, double lnv, double& psi,
                                             double& dpsi)
{
    double P = w.c[7], Q = w.d[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        P = fma(P, v, w.c[k]);
        Q = fma(Q, v, w.d[k]);
    }
    double v2 = v * v, v3 = v2 * v, v5 = v3 * v2, v6 = v3 * v3, v8 = v6 * v2;
    psi = (P + lnv * (w.cl5 * v5 + w.cl6 * v6)) / v5;
    dpsi = (Q + lnv * w.dl6 * v6) / v8;
}

// Parameter derivation (Sec. II A): masses, PN coefficients with the 1.5PN spin-orbit and
// 2PN spin-spin terms, taper/cut frequencies, f_max = argmax f^2 A, distance scaling,
// wave frame and mode factors.  theta is SoA [11][W].
__device__ inline void hm_setup(Walker& w, double q, double iota, double phi);

__device__ inline void walker_setup(const double* __restrict__ theta, int64_t W, int64_t i,
                                    Walker& w, uint32_t modes = 1u)
{
    const double mt = theta[kMT * W + i], q = theta[kQ * W + i];
    const double a1 = theta[kA1 * W + i], a2 = theta[kA2 * W + i];
    const double dl = theta[kDL * W + i], phi = theta[kPhi * W + i];
    const double iota = theta[kIota * W + i], lam = theta[kLam * W + i];
    const double bet = theta[kBeta * W + i], pol = theta[kPsi * W + i];
    const double tref = theta[kTref * W + i];

    const double opq = 1.0 + q;
    const double eta = q / (opq * opq);
    const double x1 = 1.0 / opq, x2 = q / opq;  // m_i / M
    const double M = mt * kMsunSec;
    const double dist = dl * 1e9 * kParsec / kClight;

    const double so = (113.0 / 12.0 * x1 * x1 + 25.0 / 4.0 * eta) * a1 +
                      (113.0 / 12.0 * x2 * x2 + 25.0 / 4.0 * eta) * a2;
    const double ss = 79.0 / 8.0 * eta * a1 * a2;
    const double pi2 = kPi * kPi;
    double al[8], alog5, alog6;
    al[0] = 1.0;
    al[1] = 0.0;
    al[2] = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
    al[3] = -16.0 * kPi + 4.0 * so;
    al[4] = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta - 10.0 * ss;
    al[5] = kPi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
    alog5 = 3.0 * al[5];
    al[6] = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi2 - 6848.0 / 21.0 * kEulerGamma -
            6848.0 / 21.0 * 1.386294361119890618834464242916353136 +
            eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi2) + 76055.0 / 1728.0 * eta * eta -
            127825.0 / 1296.0 * eta * eta * eta;
    alog6 = -6848.0 / 21.0;
    al[7] = kPi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta);

    const double pre = 3.0 / (128.0 * eta);
    const double dpre = kPi * M / (128.0 * eta);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        w.c[k] = pre * al[k];
        w.d[k] = dpre * ((k - 5) * al[k]);
    }
    w.d[5] += dpre * alog5;          // d/dv of alog5 ln v
    w.d[6] += dpre * alog6;          // d/dv of alog6 v ln v, non-log part
    w.cl5 = pre * alog5;
    w.cl6 = pre * alog6;
    w.dl6 = dpre * alog6;            // (k - 5) alog_k for k = 6

    w.piM = kPi * M;
    w.cbrt_piM = cbrt(w.piM);
    w.icbrt_piM = 1.0 / w.cbrt_piM;
    w.ln_cbrt_piM = log(w.piM) / 3.0;
    w.tref = tref;
    const double fc = 0.05 / M;
    w.fcut = 0.2 / M;
    w.fmax = fc * sqrt(5.0 / 12.0);
    w.inv_fc2 = 1.0 / (fc * fc);
    // A(f) = sqrt(2 pi/3) pi^{-2/3} M^{5/6} eta^{1/2} f^{-7/6} exp(-(f/fc)^2) / D, and
    // f^{-7/6} = (pi M)^{7/6} v^{-7/2}.
    w.amp = sqrt(2.0 * kPi / 3.0) * pow(kPi, -2.0 / 3.0) * pow(M, 5.0 / 6.0) * sqrt(eta) / dist *
            pow(w.piM, 7.0 / 6.0);
    {
        double v = cbrt(w.piM * w.fmax);
        double ps, dps;
        pn_phase_f64(w, v, log(v), ps, dps);
        w.psi_max = ps;
        w.dpsi_max = dps;
    }
    sincos(kTwoPi * tref / kYear, &w.sa_ref, &w.ca_ref);

    // wave frame: k = -(cos b cos l, cos b sin l, sin b); u, v transverse with u x v = k
    double sl, cl, sb, cb, s2p, c2p;
    sincos(lam, &sl, &cl);
    sincos(bet, &sb, &cb);
    sincos(2.0 * pol, &s2p, &c2p);
    const double u[3] = {sl, -cl, 0.0};
    const double vv[3] = {-sb * cl, -sb * sl, cb};
    w.k[0] = -cb * cl;
    w.k[1] = -cb * sl;
    w.k[2] = -sb;
    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        double ep = u[ii[m]] * u[jj[m]] - vv[ii[m]] * vv[jj[m]];
        double ec = u[ii[m]] * vv[jj[m]] + vv[ii[m]] * u[jj[m]];
        w.Pp[m] = c2p * ep + s2p * ec;
        w.Pc[m] = -s2p * ep + c2p * ec;
    }
    // K+ = sqrt(5/64 pi)(1 + cos^2 i) e^{2 i phi}, Kx = 2 i sqrt(5/64 pi) cos i e^{2 i phi}
    const double ylm = sqrt(5.0 / (64.0 * kPi));
    const double ci = cos(iota);
    double s2f, c2f;
    sincos(2.0 * phi, &s2f, &c2f);
    const double ap = ylm * (1.0 + ci * ci), ac = 2.0 * ylm * ci;
    w.Kp[0] = ap * c2f;
    w.Kp[1] = ap * s2f;
    w.Kc[0] = -ac * s2f;
    w.Kc[1] = ac * c2f;
    w.modes = modes;
    if (modes != 1u) hm_setup(w, q, iota, phi);
}

// Spin-weighted harmonics -2Y_{l,+-m}(iota, .) without the e^{+-i m phi} factor, written out in
// C = cos(iota/2), S = sin(iota/2) for the six modes: y[0] = -2Y_{l,m}, y[1] = -2Y_{l,-m}.
__device__ inline void hm_ylm(int b, double C, double S, double y[2])
{
    const double rpi = 0.564189583547756286948079451560772586;   // 1/sqrt(pi)
    const double C2 = C * C, S2 = S * S;
    switch (b) {
    case 0:   // (2, +-2)
        y[0] = 0.5 * 2.236067977499789696 * rpi * C2 * C2;
        y[1] = 0.5 * 2.236067977499789696 * rpi * S2 * S2;
        break;
    case 1:   // (3, +-3)
        y[0] = -0.5 * 6.480740698407860230 * rpi * C2 * C2 * C * S;
        y[1] = 0.5 * 6.480740698407860230 * rpi * C * S * S2 * S2;
        break;
    case 2:   // (4, +-4)
        y[0] = 3.0 * 2.645751311064590590 * rpi * C2 * C2 * C2 * S2;
        y[1] = 3.0 * 2.645751311064590590 * rpi * C2 * S2 * S2 * S2;
        break;
    case 3:   // (2, +-1)
        y[0] = 2.236067977499789696 * rpi * C2 * C * S;
        y[1] = 2.236067977499789696 * rpi * C * S2 * S;
        break;
    case 4:   // (3, +-2)
        y[0] = 0.5 * 2.645751311064590590 * rpi * C2 * C2 * (C2 - 5.0 * S2);
        y[1] = 0.5 * 2.645751311064590590 * rpi * S2 * S2 * (5.0 * C2 - S2);
        break;
    default:  // (4, +-3)
        y[0] = -1.5 * 3.741657386773941386 * rpi * C2 * C2 * C * S * (C2 - 3.0 * S2);
        y[1] = 1.5 * 3.741657386773941386 * rpi * C * S * S2 * S2 * (3.0 * C2 - S2);
        break;
    }
}

// Per-mode polarisation factors, positive frequencies, in the convention of the (2,2) factors
// above: K+ = (Y_lm + (-1)^l conj(Y_{l,-m}))/2, Kx = i (Y_lm - (-1)^l conj(Y_{l,-m}))/2, both
// proportional to e^{i m phi}; folded with H_lm's constant c_lm and sqrt(2/m).
__device__ inline void hm_setup(Walker& w, double q, double iota, double phi)
{
    const double eta = q / ((1.0 + q) * (1.0 + q)), delta = (1.0 - q) / (1.0 + q);
    double S, C;
    sincos(0.5 * iota, &S, &C);
#pragma unroll
    for (int b = 0; b < kHmModes; ++b) {
        const int m = hm_m(b), l = (b == 0 || b == 3) ? 2 : (b == 1 || b == 4) ? 3 : 4;
        double y[2];
        hm_ylm(b, C, S, y);
        const double sg = (l & 1) ? -1.0 : 1.0;
        const double a = 0.5 * (y[0] + sg * y[1]), bx = 0.5 * (y[0] - sg * y[1]);
        // c_lm: 22: 1; 33: -(3i/4) sqrt(15/14) delta; 44: -(8/9) sqrt(5/7)(1 - 3 eta);
        // 21: (i/3) delta; 32: (1/3) sqrt(5/7)(1 - 3 eta); 43: -(9i/(4 sqrt 70)) delta (1 - 2 eta)
        double cr = 0.0, cim = 0.0;
        switch (b) {
        case 0: cr = 1.0; break;
        case 1: cim = -0.75 * 1.035098339013531 * delta; break;
        case 2: cr = -8.0 / 9.0 * 0.845154254728516 * (1.0 - 3.0 * eta); break;
        case 3: cim = delta / 3.0; break;
        case 4: cr = 1.0 / 3.0 * 0.845154254728516 * (1.0 - 3.0 * eta); break;
        default: cim = -9.0 / (4.0 * 8.366600265340756) * delta * (1.0 - 2.0 * eta); break;
        }
        const double sc = sqrt(2.0 / m);
        cr *= sc;
        cim *= sc;
        double sm, cm;
        sincos(m * phi, &sm, &cm);
        // K+ = a e^{i m phi} c, Kx = i bx e^{i m phi} c
        const double er = cm * cr - sm * cim, ei = cm * cim + sm * cr;
        w.hk[b][0] = a * er;
        w.hk[b][1] = a * ei;
        w.hk[b][2] = -bx * ei;
        w.hk[b][3] = bx * er;
    }
}

struct cd { double re, im; };
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.re * s, a.im * s}; }

__device__ __forceinline__ double sinc_f64(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

// n.P.n for a symmetric tensor stored as (xx, xy, xz, yy, yz, zz)
__device__ __forceinline__ double nPn(const double* P, const double* n)
{
    return P[0] * n[0] * n[0] + P[3] * n[1] * n[1] + P[5] * n[2] * n[2] +
           2.0 * (P[1] * n[0] * n[1] + P[2] * n[0] * n[2] + P[4] * n[1] * n[2]);
}

// Transfer T_c(f) at orbital angle alpha (sin sa, cos ca), float64.  Rigid equilateral
// constellation: spacecraft i at offset rho (sin psi_i t^ - cos psi_i w^) from the guiding
// centre, psi_i = alpha - 2 pi i/3, t^ = (-sa, ca, 0), w^ = (ca/2, sa/2, sqrt3/2).  Each arm
// (i, j) contributes g = -i x e^{-i pi f (L + k.(o_i + o_j))} F with x = pi f L and
// F = n.(P+ K+ + Px Kx).n; link i->j adds sinc(x (1 - k.n)), link j->i sinc(x (1 + k.n)).
// First-generation TDI with D = e^{-2 i x}, then A, E, T.
__device__ inline void transfer_f64(const Walker& w, double f, double sa, double ca, const double* Kp,
                                    const double* Kc, cd T[3])
{
    const double rho = kArmSec / kSqrt3;
    // sin/cos(alpha - 2 pi i/3): cos(2pi/3) = -1/2, sin(2pi/3) = sqrt3/2
    const double sp[3] = {sa, -0.5 * sa - 0.5 * kSqrt3 * ca, -0.5 * sa + 0.5 * kSqrt3 * ca};
    const double cp[3] = {ca, -0.5 * ca + 0.5 * kSqrt3 * sa, -0.5 * ca - 0.5 * kSqrt3 * sa};
    double o[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o[i][0] = rho * (sp[i] * (-sa) - cp[i] * 0.5 * ca);
        o[i][1] = rho * (sp[i] * ca - cp[i] * 0.5 * sa);
        o[i][2] = rho * (-cp[i] * 0.5 * kSqrt3);
    }
    const double x = kPi * f * kArmSec;
    cd yf[3], yb[3];  // arm a: forward link i->j, backward j->i, arms (0,1), (1,2), (2,0)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = a, j = (a + 1) % 3;
        double n[3], kn = 0.0, ko = 0.0;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            n[m] = (o[j][m] - o[i][m]) / kArmSec;
            kn += w.k[m] * n[m];
            ko += w.k[m] * (o[i][m] + o[j][m]);
        }
        const double np = nPn(w.Pp, n), nc = nPn(w.Pc, n);
        cd F = {np * Kp[0] + nc * Kc[0], np * Kp[1] + nc * Kc[1]};
        double sph, cph;
        sincos(kPi * f * (kArmSec + ko), &sph, &cph);
        // -i x e^{-i ph} = -x (sin ph + i cos ph)
        cd g = cmul({-x * sph, -x * cph}, F);
        yf[a] = cscale(g, sinc_f64(x * (1.0 - kn)));
        yb[a] = cscale(g, sinc_f64(x * (1.0 + kn)));
    }
    const cd y12 = yf[0], y21 = yb[0], y23 = yf[1], y32 = yb[1], y31 = yf[2], y13 = yb[2];
    double sd, cdl;
    sincos(2.0 * x, &sd, &cdl);
    const cd D = {cdl, -sd};
    const cd D2 = cmul(D, D);
    const cd wf = {1.0 - D2.re, -D2.im};
    const cd X = cmul(wf, csub(cadd(y21, cmul(D, y12)), cadd(y31, cmul(D, y13))));
    const cd Y = cmul(wf, csub(cadd(y32, cmul(D, y23)), cadd(y12, cmul(D, y21))));
    const cd Z = cmul(wf, csub(cadd(y13, cmul(D, y31)), cadd(y23, cmul(D, y32))));
    T[0] = cscale(csub(Z, X), 1.0 / kSqrt2);
    T[1] = cscale(cadd(csub(X, cscale(Y, 2.0)), Z), 1.0 / kSqrt6);
    T[2] = cscale(cadd(cadd(X, Y), Z), 1.0 / kSqrt3);
}

// Full float64 template at f (Eqs. 7-9).  Returns false (and zeros) outside the support:
// f > f_cut or t(f) outside [0, t_obs].
__device__ inline bool point_f64(const Walker& w, double f, double t_obs, cd h[3])
{
    const double v = cbrt(w.piM * f);
    const double lnv = log(v);
    double psi_pn, dpsi_pn;
    pn_phase_f64(w, v, lnv, psi_pn, dpsi_pn);
    const double t = w.tref + (dpsi_pn - w.dpsi_max) * kInvTwoPi;
    if (!(f <= w.fcut) || t < 0.0 || t > t_obs) {
        h[0] = h[1] = h[2] = {0.0, 0.0};
        return false;
    }
    const double amp = w.amp * exp(-f * f * w.inv_fc2) / (v * v * v * sqrt(v));
    double sa, ca;
    sincos(kTwoPi * t / kYear, &sa, &ca);
    const double kc = kAUSec * (w.k[0] * ca + w.k[1] * sa);
    const double Phi = kTwoPi * f * (w.tref + kc) + psi_pn - w.psi_max - (f - w.fmax) * w.dpsi_max;
    double sP, cP;
    sincos(Phi, &sP, &cP);
    cd T[3];
    transfer_f64(w, f, sa, ca, w.Kp, w.Kc, T);
    const cd e = {amp * cP, -amp * sP};
    h[0] = cmul(e, T[0]);
    h[1] = cmul(e, T[1]);
    h[2] = cmul(e, T[2]);
    return true;
}

// Template of the walker's modes at f, float64: per mode the (2,2) model at f2 = 2f/m (phase
// scaled by m/2, amplitude by v^{p_lm}), the orbit and the transfer at t_lm(f), summed.
// Returns false (and zeros) when no mode is in its support.
// One mode (index b) of the walker's template at f, float64: the (2,2) model at f2 = 2f/m
// (phase scaled by m/2, amplitude by v^{p_lm}), the orbit and the transfer at t_lm(f).
// Returns false (and leaves h alone) outside the mode's support.
__device__ inline bool mode_point_f64(const Walker& w, int b, double f, double t_obs, cd h[3])
{
    const int m = hm_m(b);
    const double f2 = 2.0 * f / m;
    const double v = cbrt(w.piM * f2);
    double psi_pn, dpsi_pn;
    pn_phase_f64(w, v, log(v), psi_pn, dpsi_pn);
    const double t = w.tref + (dpsi_pn - w.dpsi_max) * kInvTwoPi;
    if (!(f2 <= w.fcut) || t < 0.0 || t > t_obs) return false;
    double amp = w.amp * exp(-f2 * f2 * w.inv_fc2) / (v * v * v * sqrt(v));
    for (int j = 0; j < hm_vpow(b); ++j) amp *= v;
    double sa, ca;
    sincos(kTwoPi * t / kYear, &sa, &ca);
    const double kc = kAUSec * (w.k[0] * ca + w.k[1] * sa);
    const double Phi = 0.5 * m * (kTwoPi * f2 * w.tref + psi_pn - w.psi_max - (f2 - w.fmax) * w.dpsi_max) +
                       kTwoPi * f * kc;
    double sP, cP;
    sincos(Phi, &sP, &cP);
    cd T[3];
    transfer_f64(w, f, sa, ca, &w.hk[b][0], &w.hk[b][2], T);
    const cd e = {amp * cP, -amp * sP};
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = cmul(e, T[c]);
    return true;
}

// Template of the walker's modes at f, float64: the modes of mode_point_f64, summed.
// Returns false (and zeros) when no mode is in its support.
__device__ inline bool point_hm_f64(const Walker& w, double f, double t_obs, cd h[3])
{
    h[0] = h[1] = h[2] = {0.0, 0.0};
    bool any = false;
    for (int b = 0; b < kHmModes; ++b) {
        if (!(w.modes & (1u << b))) continue;
        cd hb[3];
        if (!mode_point_f64(w, b, f, t_obs, hb)) continue;
        any = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) h[c] = cadd(h[c], hb[c]);
    }
    return any;
}

// The walker's template, whatever its modes (W0 for the (2,2) mode alone).
__device__ __forceinline__ bool point_model_f64(const Walker& w, double f, double t_obs, cd h[3])
{
    return w.modes == 1u ? point_f64(w, f, t_obs, h) : point_hm_f64(w, f, t_obs, h);
}

// Support test alone (band search): t(f) and the cut, float64.
__device__ inline bool support_f64(const Walker& w, double f, double t_obs)
{
    const double v = cbrt(w.piM * f);
    double psi_pn, dpsi_pn;
    pn_phase_f64(w, v, log(v), psi_pn, dpsi_pn);
    const double t = w.tref + (dpsi_pn - w.dpsi_max) * kInvTwoPi;
    return (f <= w.fcut) && t >= 0.0 && t <= t_obs;
}

// Some mode of the walker is in its support at f (the (2,2) mode at f2 = 2f/m).
__device__ inline bool support_model_f64(const Walker& w, double f, double t_obs)
{
    if (w.modes == 1u) return support_f64(w, f, t_obs);
    for (int b = 0; b < kHmModes; ++b)
        if ((w.modes & (1u << b)) && support_f64(w, 2.0 * f / hm_m(b), t_obs)) return true;
    return false;
}

}  // namespace mbh

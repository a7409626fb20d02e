/*
 * FP64 CPU oracle for the batched LISA likelihood of massive-black-hole-binary
 * templates (Katz, arXiv:2111.01064, Sec. II).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA library, and it never reads a value
 * that the CUDA library produced.
 *
 * Everything is plain double precision: literal loops over the grid, sums taken
 * sequentially in grid order (plus a Neumaier-compensated inner product used to
 * bound the oracle's own round-off).  OpenMP only splits independent templates
 * or walkers across threads; the arithmetic of each one is unchanged.
 *
 * What each part follows:
 *   W0 waveform       Sec. II A, Eq. 7 (A e^{-i phi}) and the f_ref = f_max
 *                     convention; PhenomD's calibration tables are not available,
 *                     so the amplitude/phase model is the stand-in "W0": TaylorF2
 *                     3.5PN phase with 1.5PN spin-orbit and 2PN spin-spin terms,
 *                     a Gaussian-tapered f^{-7/6} amplitude, t_ref/phi pinned at
 *                     f_max = argmax f^2 A.  (Parity with PhenomD itself is
 *                     unpinned; the model is pinned internally, see the tests.)
 *   t(f)              Sec. II A, Eq. 8 (SPA time-frequency map), with the sign of
 *                     the FT convention h~(f) = int h(t) e^{-2 pi i f t} dt.
 *   R0 response       Sec. II A, Eqs. 4-6 and 9: rigid equal-arm constellation,
 *                     one-link frequency-domain kernel at t(f), first-generation
 *                     TDI X, Y, Z, then A, E, T.  The transfer function of the
 *                     cited literature is not in the paper; R0 is derived here
 *                     from the time-domain one-link Doppler response.
 *   PSD               Sec. II, Eq. 3 remark (A = E != T): analytic first-
 *                     generation TDI noise with acceleration 3e-15 m/s^2/rtHz and
 *                     OMS 15e-12 m/rtHz, L = 2.5e9 m.
 *   inner product     Sec. II, Eq. 3 (sum over A, E, T and the grid, times df).
 *   log-likelihood    Sec. II, Eq. 2 (no normalisation constant; <d|d> included).
 *   heterodyne        Sec. II B, Eqs. 10-19 and Sec. III B (log-spaced bins over
 *                     the band where h0 != 0): summary data A0, A1, B0, B1 per bin
 *                     and channel, bin centre f_b, r = h/h0 linear in each bin.
 *   higher harmonics  Sec. II A, Eqs. 7-9 (template = sum over (l,m) of the transfer at
 *                     t_lm(f) times h_lm): the stand-in "W0-HM" for PhenomHM with the
 *                     modes (2,2), (3,3), (4,4), (2,1), (3,2), (4,3).  Mode (l,m) takes
 *                     the (2,2) phase at 2f/m scaled by m/2 (so t_lm(f) = t_22(2f/m),
 *                     Eq. 8), the (2,2) amplitude at 2f/m times sqrt(2/m) (the SPA
 *                     factor of a harmonic m of the same orbital phase) and the
 *                     leading post-Newtonian mode factor H_lm(x) of Blanchet, Faye, Iyer
 *                     & Sinha (2008); polarisations from the spin-weighted harmonics
 *                     -2Y_lm (Goldberg et al. 1967).  Parity with PhenomHM itself is
 *                     unpinned.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---- constants ---------------------------------------------------------- */
#define O_PI 3.14159265358979323846
#define O_MTSUN 4.925490947641267e-6   /* G Msun / c^3 [s] */
#define O_C 299792458.0                /* speed of light [m/s] */
#define O_PC 3.085677581491367e16      /* parsec [m] */
#define O_AU 1.495978707e11            /* astronomical unit [m] */
#define O_YEAR 31557600.0              /* Julian year [s] */
#define O_LARM 2.5e9                   /* arm length [m] */
#define O_GAMMA_E 0.5772156649015329   /* Euler's constant */

enum { P_MT, P_Q, P_A1, P_A2, P_DL, P_PHI, P_IOTA, P_LAM, P_BETA, P_PSI, P_TREF };

/* ========================================================================== */
/* W0: amplitude and phase of the (2,2) mode (Sec. II A, Eq. 7)                */
/* ========================================================================== */
typedef struct {
    double M;            /* total mass in seconds */
    double eta;          /* symmetric mass ratio */
    double dist;         /* luminosity distance in seconds */
    double tref;         /* t(f_max) */
    double fc, fcut, fmax;
    double amp0;         /* A(f) = amp0 f^{-7/6} exp(-(f/fc)^2) inside the support */
    double alpha[8];     /* TaylorF2 coefficients of v^k */
    double alpha_log[8]; /* coefficients of v^k ln v */
    double psi_max;      /* Psi_PN(f_max) */
    double dpsi_max;     /* dPsi_PN/df at f_max */
} w0_t;

static double psi_pn(const w0_t* w, double f)
{
    /* Psi_PN = 3/(128 eta v^5) sum_k (alpha_k + alpha_log_k ln v) v^k */
    double v = cbrt(O_PI * w->M * f);
    double lv = log(v);
    double s = 0.0;
    for (int k = 0; k < 8; ++k)
        s += (w->alpha[k] + w->alpha_log[k] * lv) * pow(v, k);
    return 3.0 / (128.0 * w->eta * pow(v, 5)) * s;
}

static double dpsi_pn(const w0_t* w, double f)
{
    /* d/df of psi_pn: dv/df = pi M / (3 v^2), so
       dPsi/df = pi M/(128 eta) sum_k [(k-5)(alpha_k + alpha_log_k ln v) + alpha_log_k] v^{k-8} */
    double v = cbrt(O_PI * w->M * f);
    double lv = log(v);
    double s = 0.0;
    for (int k = 0; k < 8; ++k)
        s += ((k - 5) * (w->alpha[k] + w->alpha_log[k] * lv) + w->alpha_log[k]) * pow(v, k - 8);
    return O_PI * w->M / (128.0 * w->eta) * s;
}

static void w0_setup(const double* th, w0_t* w)
{
    double mt = th[P_MT], q = th[P_Q];
    double d1 = 1.0 / (1.0 + q), d2 = q / (1.0 + q);   /* m_i / M_T */
    double eta = q / ((1.0 + q) * (1.0 + q));
    double a1 = th[P_A1], a2 = th[P_A2];
    double pi = O_PI;

    w->M = mt * O_MTSUN;
    w->eta = eta;
    w->dist = th[P_DL] * 1e9 * O_PC / O_C;
    w->tref = th[P_TREF];

    /* spin-orbit (1.5PN) and spin-spin (2PN) combinations */
    double beta = (113.0 / 12.0 * d1 * d1 + 25.0 / 4.0 * eta) * a1
                + (113.0 / 12.0 * d2 * d2 + 25.0 / 4.0 * eta) * a2;
    double sigma = 79.0 / 8.0 * eta * a1 * a2;

    for (int k = 0; k < 8; ++k) { w->alpha[k] = 0.0; w->alpha_log[k] = 0.0; }
    w->alpha[0] = 1.0;
    w->alpha[1] = 0.0;
    w->alpha[2] = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
    w->alpha[3] = -16.0 * pi + 4.0 * beta;
    w->alpha[4] = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta
                - 10.0 * sigma;
    /* 2.5PN: pi (38645/756 - 65/9 eta)(1 + 3 ln v); the constant part only shifts
       the phase by a constant, which the f_max pinning removes */
    w->alpha[5] = pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
    w->alpha_log[5] = 3.0 * pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
    /* 3PN, with ln(4v) = ln 4 + ln v */
    w->alpha[6] = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi
                - 6848.0 / 21.0 * O_GAMMA_E - 6848.0 / 21.0 * log(4.0)
                + eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi)
                + 76055.0 / 1728.0 * eta * eta - 127825.0 / 1296.0 * eta * eta * eta;
    w->alpha_log[6] = -6848.0 / 21.0;
    w->alpha[7] = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta
                        - 74045.0 / 756.0 * eta * eta);

    w->fc = 0.05 / w->M;
    w->fcut = 0.2 / w->M;
    /* f^2 A ~ f^{5/6} exp(-(f/fc)^2) is largest where 5/(6f) = 2f/fc^2 */
    w->fmax = w->fc * sqrt(5.0 / 12.0);
    /* (2,2) amplitude normalised so that with the -2Y22 factor of the response
       the Newtonian h+ amplitude is sqrt(5/24) pi^{-2/3} Mc^{5/6} f^{-7/6} / D */
    w->amp0 = sqrt(2.0 * pi / 3.0) * pow(pi, -2.0 / 3.0) * pow(w->M, 5.0 / 6.0)
            * sqrt(eta) / w->dist;
    w->psi_max = psi_pn(w, w->fmax);
    w->dpsi_max = dpsi_pn(w, w->fmax);
}

/* Phase Psi(f) = 2 pi f t_ref + Psi_PN(f) - Psi_PN(fmax) - (f - fmax) Psi_PN'(fmax),
   so that t(f) = Psi'(f)/(2 pi) equals t_ref at f_max. */
static double w0_phase(const w0_t* w, double f)
{
    return 2.0 * O_PI * f * w->tref + psi_pn(w, f) - w->psi_max - (f - w->fmax) * w->dpsi_max;
}

static double w0_time(const w0_t* w, double f)
{
    return w->tref + (dpsi_pn(w, f) - w->dpsi_max) / (2.0 * O_PI);
}

/* Amplitude; zero above f_cut and where the track t(f) lies outside [0, t_obs]. */
static double w0_amp(const w0_t* w, double f, double t, double t_obs)
{
    if (!(f > 0.0) || f > w->fcut || t < 0.0 || t > t_obs) return 0.0;
    return w->amp0 * pow(f, -7.0 / 6.0) * exp(-(f / w->fc) * (f / w->fc));
}

void oracle_w0(const double* th, double t_obs, const double* f, long n,
               double* amp, double* psi, double* tf)
{
    w0_t w;
    w0_setup(th, &w);
    for (long i = 0; i < n; ++i) {
        double t = w0_time(&w, f[i]);
        tf[i] = t;
        psi[i] = w0_phase(&w, f[i]);
        amp[i] = w0_amp(&w, f[i], t, t_obs);
    }
}

/* out = [M, eta, fc, fcut, fmax, psi_max, dpsi_max, amp0, dist, alpha[0..7], alpha_log[0..7]] */
void oracle_w0_info(const double* th, double* out)
{
    w0_t w;
    w0_setup(th, &w);
    out[0] = w.M; out[1] = w.eta; out[2] = w.fc; out[3] = w.fcut; out[4] = w.fmax;
    out[5] = w.psi_max; out[6] = w.dpsi_max; out[7] = w.amp0; out[8] = w.dist;
    for (int k = 0; k < 8; ++k) { out[9 + k] = w.alpha[k]; out[17 + k] = w.alpha_log[k]; }
}

/* ========================================================================== */
/* R0: LISA response (Sec. II A, Eqs. 4-6, 9)                                  */
/* ========================================================================== */

/* Spacecraft positions in seconds at time t: guiding centre on a 1 AU circle at
   alpha = 2 pi t / yr; rigid equilateral triangle of side L in the plane spanned
   by the tangent t^ and w^ = r^/2 + sqrt(3) z^/2 (60 degrees to the ecliptic),
   circumradius L/sqrt(3), spacecraft i at angle alpha - 2 pi i/3 in that plane.
   p[3*i + j] = coordinate j of spacecraft i (i = 0, 1, 2 for spacecraft 1, 2, 3). */
void oracle_orbit(double t, double* p)
{
    double a = 2.0 * O_PI * t / O_YEAR;
    double R = O_AU / O_C;
    double rho = O_LARM / O_C / sqrt(3.0);
    double rhat[3] = { cos(a), sin(a), 0.0 };
    double that[3] = { -sin(a), cos(a), 0.0 };
    double what[3] = { 0.5 * cos(a), 0.5 * sin(a), sqrt(3.0) / 2.0 };
    for (int i = 0; i < 3; ++i) {
        double psi = a - 2.0 * O_PI * i / 3.0;
        for (int j = 0; j < 3; ++j)
            p[3 * i + j] = R * rhat[j] + rho * (sin(psi) * that[j] - cos(psi) * what[j]);
    }
}

/* Wave frame.  Propagation k = -(cos b cos l, cos b sin l, sin b); u, v span the
   transverse plane with u x v = k; polarisation tensors rotated by psi:
   P+ = cos2psi (uu - vv) + sin2psi (uv + vu), Px = -sin2psi (uu - vv) + cos2psi (uv + vu).
   Mode factors for h~+ = K+ h~22, h~x = Kx h~22 (positive frequencies, (2,+-2)
   spin-weighted harmonics): K+ = sqrt(5/64pi)(1 + cos^2 i) e^{2i phi},
   Kx = 2i sqrt(5/64pi) cos i e^{2i phi}. */
void oracle_wave_frame(const double* th, double* k, double* Pp, double* Pc,
                       double* Kp, double* Kc)
{
    double lam = th[P_LAM], bet = th[P_BETA], psi = th[P_PSI];
    double u[3] = { sin(lam), -cos(lam), 0.0 };
    double v[3] = { -sin(bet) * cos(lam), -sin(bet) * sin(lam), cos(bet) };
    k[0] = -cos(bet) * cos(lam);
    k[1] = -cos(bet) * sin(lam);
    k[2] = -sin(bet);
    double c2 = cos(2.0 * psi), s2 = sin(2.0 * psi);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double ep = u[i] * u[j] - v[i] * v[j];
            double ec = u[i] * v[j] + v[i] * u[j];
            Pp[3 * i + j] = c2 * ep + s2 * ec;
            Pc[3 * i + j] = -s2 * ep + c2 * ec;
        }
    double ci = cos(th[P_IOTA]);
    double y = sqrt(5.0 / (64.0 * O_PI));
    cplx e2 = cexp(2.0 * I * th[P_PHI]);
    cplx kp = y * (1.0 + ci * ci) * e2;
    cplx kc = 2.0 * I * y * ci * e2;
    Kp[0] = creal(kp); Kp[1] = cimag(kp);
    Kc[0] = creal(kc); Kc[1] = cimag(kc);
}

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* One-link frequency-domain kernel (frozen constellation).  From the time-domain
   Doppler response of the link s -> r,
     y(t) = [n.H(t - L - k.p_s).n - n.H(t - k.p_r).n] / (2 (1 - k.n)),
   with n = (p_r - p_s)/L, the Fourier transform gives y~(f) = G(f) n.H~(f).n with
     G = -i pi f L sinc(pi f L (1 - k.n)) exp(-i pi f (L + k.(p_s + p_r))).
   Positions in seconds. */
static cplx link_kernel(double f, const double* k, const double* ps, const double* pr)
{
    double L = O_LARM / O_C;
    double n[3], kn = 0.0, kp = 0.0;
    for (int j = 0; j < 3; ++j) {
        n[j] = (pr[j] - ps[j]) / L;
        kn += k[j] * n[j];
        kp += k[j] * (ps[j] + pr[j]);
    }
    return -I * O_PI * f * L * sinc(O_PI * f * L * (1.0 - kn)) * cexp(-I * O_PI * f * (L + kp));
}

void oracle_link(double f, const double* k, const double* ps, const double* pr, double* G)
{
    cplx g = link_kernel(f, k, ps, pr);
    G[0] = creal(g); G[1] = cimag(g);
}

/* Time-domain one-link response for a monochromatic plane wave
   h+(t) = Re(ap e^{2 pi i f0 t}), hx(t) = Re(ac e^{2 pi i f0 t}) and a frozen
   constellation: the definition that link_kernel is derived from. */
void oracle_link_td(const double* k, const double* Pp, const double* Pc,
                    const double* ps, const double* pr, double f0,
                    const double* ap, const double* ac, const double* t, long nt, double* y)
{
    double L = O_LARM / O_C;
    double n[3], kn = 0.0, kps = 0.0, kpr = 0.0;
    for (int j = 0; j < 3; ++j) {
        n[j] = (pr[j] - ps[j]) / L;
        kn += k[j] * n[j];
        kps += k[j] * ps[j];
        kpr += k[j] * pr[j];
    }
    double nPpn = 0.0, nPcn = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            nPpn += n[i] * Pp[3 * i + j] * n[j];
            nPcn += n[i] * Pc[3 * i + j] * n[j];
        }
    cplx Ap = ap[0] + I * ap[1], Ac = ac[0] + I * ac[1];
    for (long i = 0; i < nt; ++i) {
        double te = t[i] - L - kps;   /* emission, retarded to the SSB origin */
        double tr = t[i] - kpr;       /* reception */
        double hpe = creal(Ap * cexp(2.0 * I * O_PI * f0 * te));
        double hce = creal(Ac * cexp(2.0 * I * O_PI * f0 * te));
        double hpr = creal(Ap * cexp(2.0 * I * O_PI * f0 * tr));
        double hcr = creal(Ac * cexp(2.0 * I * O_PI * f0 * tr));
        y[i] = ((nPpn * hpe + nPcn * hce) - (nPpn * hpr + nPcn * hcr)) / (2.0 * (1.0 - kn));
    }
}

/* Link order used for y[6]: 1->2, 2->1, 2->3, 3->2, 3->1, 1->3. */
static const int LINK_S[6] = { 0, 1, 1, 2, 2, 0 };
static const int LINK_R[6] = { 1, 0, 2, 1, 0, 2 };

/* First-generation TDI for equal arms, delay D = exp(-2 pi i f L):
     X = (1 - D^2) [(y21 + D y12) - (y31 + D y13)]
     Y = (1 - D^2) [(y32 + D y23) - (y12 + D y21)]
     Z = (1 - D^2) [(y13 + D y31) - (y23 + D y32)]
   (y_sr = link s -> r), then A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6,
   T = (X + Y + Z)/sqrt3 (Sec. II A, Eqs. 4-6). */
static void tdi(double f, const cplx* y, cplx* xyz, cplx* aet)
{
    double L = O_LARM / O_C;
    cplx D = cexp(-2.0 * I * O_PI * f * L);
    cplx y12 = y[0], y21 = y[1], y23 = y[2], y32 = y[3], y31 = y[4], y13 = y[5];
    cplx w = 1.0 - D * D;
    cplx X = w * ((y21 + D * y12) - (y31 + D * y13));
    cplx Y = w * ((y32 + D * y23) - (y12 + D * y21));
    cplx Z = w * ((y13 + D * y31) - (y23 + D * y32));
    xyz[0] = X; xyz[1] = Y; xyz[2] = Z;
    aet[0] = (Z - X) / sqrt(2.0);
    aet[1] = (X - 2.0 * Y + Z) / sqrt(6.0);
    aet[2] = (X + Y + Z) / sqrt(3.0);
}

/* y: 6 complex (12 doubles); out: X, Y, Z, A, E, T (12 doubles) */
void oracle_tdi(double f, const double* y, double* out)
{
    cplx yy[6], xyz[3], aet[3];
    for (int l = 0; l < 6; ++l) yy[l] = y[2 * l] + I * y[2 * l + 1];
    tdi(f, yy, xyz, aet);
    for (int c = 0; c < 3; ++c) {
        out[2 * c] = creal(xyz[c]); out[2 * c + 1] = cimag(xyz[c]);
        out[6 + 2 * c] = creal(aet[c]); out[6 + 2 * c + 1] = cimag(aet[c]);
    }
}

/* A, E, T template at frequency f (Eq. 9 with the single (2,2) mode).  h[c]
   receives channel c; when xyz is non-null it receives X, Y, Z. */
static void template_point(const w0_t* w, const double* k, const double* Pp, const double* Pc,
                           cplx Kp, cplx Kc, double t_obs, double f, cplx* h, cplx* xyz_out)
{
    double t = w0_time(w, f);
    double A = w0_amp(w, f, t, t_obs);
    if (A == 0.0) {
        for (int c = 0; c < 3; ++c) { h[c] = 0.0; if (xyz_out) xyz_out[c] = 0.0; }
        return;
    }
    cplx h22 = A * cexp(-I * w0_phase(w, f));
    double p[9];
    oracle_orbit(t, p);
    cplx y[6];
    for (int l = 0; l < 6; ++l) {
        const double* ps = p + 3 * LINK_S[l];
        const double* pr = p + 3 * LINK_R[l];
        double L = O_LARM / O_C, n[3];
        for (int j = 0; j < 3; ++j) n[j] = (pr[j] - ps[j]) / L;
        double nPpn = 0.0, nPcn = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                nPpn += n[i] * Pp[3 * i + j] * n[j];
                nPcn += n[i] * Pc[3 * i + j] * n[j];
            }
        y[l] = link_kernel(f, k, ps, pr) * (nPpn * Kp + nPcn * Kc) * h22;
    }
    cplx xyz[3];
    tdi(f, y, xyz, h);
    if (xyz_out) for (int c = 0; c < 3; ++c) xyz_out[c] = xyz[c];
}

/* ---- higher harmonics ("W0-HM") ------------------------------------------ */
/* Mode b of a mode mask: bit b selects (l, m) = (HM_L[b], HM_M[b]); mask 1 = (2,2) only. */
static const int HM_L[6] = { 2, 3, 4, 2, 3, 4 };
static const int HM_M[6] = { 2, 3, 4, 1, 2, 3 };

static double factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

static double binomial(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    return factorial(n) / (factorial(k) * factorial(n - k));
}

/* Spin-weighted spherical harmonic sY_lm(theta, phi), Goldberg et al. (1967):
   (-1)^m sqrt[(l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)] sin^{2l}(theta/2)
   sum_r C(l-s, r) C(l+s, r+s-m) (-1)^{l-r-s} cot^{2r+s-m}(theta/2) e^{i m phi},
   written with cos and sin of theta/2 so that the poles need no special case. */
static cplx sylm(int s, int l, int m, double theta, double phi)
{
    double c = cos(0.5 * theta), sn = sin(0.5 * theta);
    double pre = ((m % 2) ? -1.0 : 1.0)
               * sqrt(factorial(l + m) * factorial(l - m) * (2 * l + 1)
                      / (4.0 * O_PI * factorial(l + s) * factorial(l - s)));
    double sum = 0.0;
    for (int r = 0; r <= l - s; ++r) {
        int j = r + s - m;
        if (j < 0 || j > l + s) continue;
        int pc = 2 * r + s - m;            /* power of cos(theta/2) */
        int ps = 2 * l - pc;               /* power of sin(theta/2) */
        double sign = ((l - r - s) % 2) ? -1.0 : 1.0;
        sum += binomial(l - s, r) * binomial(l + s, j) * sign * pow(c, pc) * pow(sn, ps);
    }
    return pre * sum * cexp(I * m * phi);
}

void oracle_sylm(int s, int l, int m, double theta, double phi, double* out)
{
    cplx y = sylm(s, l, m, theta, phi);
    out[0] = creal(y); out[1] = cimag(y);
}

/* Leading post-Newtonian mode factor H_lm(x) relative to the (2,2) mode (Blanchet, Faye,
   Iyer & Sinha 2008), x = (pi M f_orb 2)^{2/3}, delta = (m1 - m2)/M. */
static cplx hm_hhat(int b, double eta, double delta, double x)
{
    switch (b) {
    case 0: return 1.0;
    case 1: return -0.75 * I * sqrt(15.0 / 14.0) * delta * sqrt(x);
    case 2: return -8.0 / 9.0 * sqrt(5.0 / 7.0) * (1.0 - 3.0 * eta) * x;
    case 3: return I / 3.0 * delta * sqrt(x);
    case 4: return 1.0 / 3.0 * sqrt(5.0 / 7.0) * (1.0 - 3.0 * eta) * x;
    default: return -9.0 * I / (4.0 * sqrt(70.0)) * delta * (1.0 - 2.0 * eta) * pow(x, 1.5);
    }
}

/* Polarisation factors of mode b (positive frequencies, in the convention of the (2,2)
   factors above): K+ = (Y_lm + (-1)^l conj(Y_{l,-m}))/2, Kx = i (Y_lm - (-1)^l conj(Y_{l,-m}))/2,
   Y = -2Y(iota, phi_ref). */
static void hm_factors(int b, double iota, double phi, cplx* Kp, cplx* Kc)
{
    int l = HM_L[b], m = HM_M[b];
    cplx y = sylm(-2, l, m, iota, phi), ym = conj(sylm(-2, l, -m, iota, phi));
    double sg = (l % 2) ? -1.0 : 1.0;
    *Kp = 0.5 * (y + sg * ym);
    *Kc = 0.5 * I * (y - sg * ym);
}

/* Mode b alone: |h_lm|, Psi_lm and t_lm at f (zero amplitude outside its support). */
static void hm_mode(const w0_t* w, double eta, double delta, int b, double t_obs, double f,
                    double* amp, double* psi, double* t, cplx* H)
{
    int m = HM_M[b];
    double f2 = 2.0 * f / m;
    *t = w0_time(w, f2);
    double a = w0_amp(w, f2, *t, t_obs);
    double x = pow(O_PI * w->M * f2, 2.0 / 3.0);
    *H = hm_hhat(b, eta, delta, x);
    *amp = a * sqrt(2.0 / m);
    *psi = 0.5 * m * w0_phase(w, f2);
}

/* Template of the selected modes at f: per mode the transfer at t_lm(f) (orbit positions
   at t_lm), summed over modes link by link; TDI is linear, so it is applied once. */
static void template_point_hm(const w0_t* w, const double* th, const double* k, const double* Pp,
                              const double* Pc, unsigned modes, double t_obs, double f, cplx* h,
                              cplx* xyz_out)
{
    double q = th[P_Q];
    double eta = q / ((1.0 + q) * (1.0 + q)), delta = (1.0 - q) / (1.0 + q);
    cplx y[6] = { 0, 0, 0, 0, 0, 0 };
    int any = 0;
    for (int b = 0; b < 6; ++b) {
        if (!(modes & (1u << b))) continue;
        double amp, psi, t;
        cplx H;
        hm_mode(w, eta, delta, b, t_obs, f, &amp, &psi, &t, &H);
        if (amp == 0.0) continue;
        any = 1;
        cplx Kp, Kc;
        hm_factors(b, th[P_IOTA], th[P_PHI], &Kp, &Kc);
        cplx hlm = amp * H * cexp(-I * psi);
        double p[9];
        oracle_orbit(t, p);
        for (int l = 0; l < 6; ++l) {
            const double* ps = p + 3 * LINK_S[l];
            const double* pr = p + 3 * LINK_R[l];
            double L = O_LARM / O_C, n[3];
            for (int j = 0; j < 3; ++j) n[j] = (pr[j] - ps[j]) / L;
            double nPpn = 0.0, nPcn = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    nPpn += n[i] * Pp[3 * i + j] * n[j];
                    nPcn += n[i] * Pc[3 * i + j] * n[j];
                }
            y[l] += link_kernel(f, k, ps, pr) * (nPpn * Kp + nPcn * Kc) * hlm;
        }
    }
    if (!any) {
        for (int c = 0; c < 3; ++c) { h[c] = 0.0; if (xyz_out) xyz_out[c] = 0.0; }
        return;
    }
    cplx xyz[3];
    tdi(f, y, xyz, h);
    if (xyz_out) for (int c = 0; c < 3; ++c) xyz_out[c] = xyz[c];
}

/* Template h[c*n + i] (complex, interleaved re/im) at frequencies f[0..n) for the modes
   of the mask (1 = the (2,2) mode: W0). */
static void template_eval_modes(const double* th, double t_obs, const double* f, long n,
                                unsigned modes, cplx* h, cplx* xyz)
{
    w0_t w;
    w0_setup(th, &w);
    double k[3], Pp[9], Pc[9], kp[2], kc[2];
    oracle_wave_frame(th, k, Pp, Pc, kp, kc);
    cplx Kp = kp[0] + I * kp[1], Kc = kc[0] + I * kc[1];
    for (long i = 0; i < n; ++i) {
        cplx hh[3], xx[3];
        if (modes == 1u)
            template_point(&w, k, Pp, Pc, Kp, Kc, t_obs, f[i], hh, xx);
        else
            template_point_hm(&w, th, k, Pp, Pc, modes, t_obs, f[i], hh, xx);
        for (int c = 0; c < 3; ++c) {
            h[c * n + i] = hh[c];
            if (xyz) xyz[c * n + i] = xx[c];
        }
    }
}

static void template_eval(const double* th, double t_obs, const double* f, long n, cplx* h,
                          cplx* xyz)
{
    template_eval_modes(th, t_obs, f, n, 1u, h, xyz);
}

/* Mode b alone on frequencies f: amp, psi, t (the SPA relations are pinned with these). */
void oracle_hm_mode(const double* th, double t_obs, const double* f, long n, int b, double* amp,
                    double* psi, double* tf, double* hre, double* him)
{
    w0_t w;
    w0_setup(th, &w);
    double q = th[P_Q];
    double eta = q / ((1.0 + q) * (1.0 + q)), delta = (1.0 - q) / (1.0 + q);
    for (long i = 0; i < n; ++i) {
        cplx H;
        hm_mode(&w, eta, delta, b, t_obs, f[i], amp + i, psi + i, tf + i, &H);
        hre[i] = creal(H);
        him[i] = cimag(H);
    }
}

void oracle_template_hm(const double* th, double t_obs, const double* f, long n, unsigned modes,
                        double* h)
{
    template_eval_modes(th, t_obs, f, n, modes, (cplx*)h, NULL);
}

void oracle_template(const double* th, double t_obs, const double* f, long n, double* h)
{
    template_eval(th, t_obs, f, n, (cplx*)h, NULL);
}

void oracle_template_xyz(const double* th, double t_obs, const double* f, long n, double* h,
                         double* xyz)
{
    template_eval(th, t_obs, f, n, (cplx*)h, (cplx*)xyz);
}

/* Gather one column of an SoA [11][W] parameter array. */
static void theta_col(const double* th, long W, long i, double* out)
{
    for (int j = 0; j < 11; ++j) out[j] = th[j * W + i];
}

/* Batch on the grid f_k = f0 + k df: h[(w*3 + c)*n + k], modes of the mask. */
void oracle_template_batch_hm(const double* th, long W, double f0, double df, long n,
                              double t_obs, unsigned modes, double* h)
{
    double* f = malloc(sizeof(double) * n);
    for (long k = 0; k < n; ++k) f[k] = f0 + k * df;
#pragma omp parallel for schedule(dynamic)
    for (long i = 0; i < W; ++i) {
        double t[11];
        theta_col(th, W, i, t);
        template_eval_modes(t, t_obs, f, n, modes, (cplx*)h + i * 3 * n, NULL);
    }
    free(f);
}

void oracle_template_batch(const double* th, long W, double f0, double df, long n,
                           double t_obs, double* h)
{
    oracle_template_batch_hm(th, W, f0, df, n, t_obs, 1u, h);
}

/* ========================================================================== */
/* Noise PSD (Sec. II, remark under Eq. 3)                                     */
/* ========================================================================== */
/* x = 2 pi f L/c;
   S_acc = (3e-15)^2 (1 + (4e-4/f)^2)(1 + (f/8e-3)^4) / (2 pi f c)^2
   S_oms = (15e-12)^2 (1 + (2e-3/f)^4) (2 pi f / c)^2
   S_A = S_E = 8 sin^2 x [2 S_acc (3 + 2 cos x + cos 2x) + S_oms (2 + cos x)]
   S_T = 32 sin^2 x sin^2(x/2) [4 S_acc sin^2(x/2) + S_oms]
   S[c*n + i], channels A, E, T. */
void oracle_psd(const double* f, long n, double* S)
{
    for (long i = 0; i < n; ++i) {
        double fi = f[i];
        double x = 2.0 * O_PI * fi * O_LARM / O_C;
        double sacc = 3e-15 * 3e-15 * (1.0 + pow(4e-4 / fi, 2)) * (1.0 + pow(fi / 8e-3, 4))
                    / pow(2.0 * O_PI * fi * O_C, 2);
        double soms = 15e-12 * 15e-12 * (1.0 + pow(2e-3 / fi, 4)) * pow(2.0 * O_PI * fi / O_C, 2);
        double sx = sin(x), sh = sin(0.5 * x);
        double sa = 8.0 * sx * sx * (2.0 * sacc * (3.0 + 2.0 * cos(x) + cos(2.0 * x))
                                     + soms * (2.0 + cos(x)));
        double st = 32.0 * sx * sx * sh * sh * (4.0 * sacc * sh * sh + soms);
        S[i] = sa;
        S[n + i] = sa;
        S[2 * n + i] = st;
    }
}

/* ========================================================================== */
/* Inner product and direct log-likelihood (Sec. II, Eqs. 2-3)                 */
/* ========================================================================== */
/* <a|b> = 4 Re sum_{c in A,E,T} sum_k conj(a_ck) b_ck / S_ck df.  a, b, S are
   [3][n] (complex interleaved for a, b).  compensated != 0 uses Neumaier
   summation. */
double oracle_inner(const double* a, const double* b, const double* S, long n, double df,
                    int compensated)
{
    const cplx* ca = (const cplx*)a;
    const cplx* cb = (const cplx*)b;
    double s = 0.0, comp = 0.0;
    for (int c = 0; c < 3; ++c)
        for (long k = 0; k < n; ++k) {
            double term = 4.0 * creal(conj(ca[c * n + k]) * cb[c * n + k]) / S[c * n + k] * df;
            if (compensated) {
                double t = s + term;
                if (fabs(s) >= fabs(term)) comp += (s - t) + term;
                else comp += (term - t) + s;
                s = t;
            } else {
                s += term;
            }
        }
    return s + comp;
}

/* Direct likelihood for W templates against data d ([3][n] complex) on the grid
   f_k = f0 + k df, k in [0, n): out[0*W + i] = lnL, out[W + i] = <d|h>,
   out[2W + i] = <h|h>, with lnL = -1/2 (<d|d> + <h|h> - 2 <d|h>). */
void oracle_direct_hm(const double* th, long W, double f0, double df, long n, double t_obs,
                      unsigned modes, const double* d, const double* S, double* out)
{
    double dd = oracle_inner(d, d, S, n, df, 0);
    double* f = malloc(sizeof(double) * n);
    for (long k = 0; k < n; ++k) f[k] = f0 + k * df;
#pragma omp parallel for schedule(dynamic)
    for (long i = 0; i < W; ++i) {
        double t[11];
        theta_col(th, W, i, t);
        cplx* h = malloc(sizeof(cplx) * 3 * n);
        template_eval_modes(t, t_obs, f, n, modes, h, NULL);
        double dh = oracle_inner(d, (const double*)h, S, n, df, 0);
        double hh = oracle_inner((const double*)h, (const double*)h, S, n, df, 0);
        out[i] = -0.5 * (dd + hh - 2.0 * dh);
        out[W + i] = dh;
        out[2 * W + i] = hh;
        free(h);
    }
    free(f);
}

void oracle_direct(const double* th, long W, double f0, double df, long n, double t_obs,
                   const double* d, const double* S, double* out)
{
    oracle_direct_hm(th, W, f0, df, n, t_obs, 1u, d, S, out);
}

/* ========================================================================== */
/* Heterodyned likelihood (Sec. II B, Eqs. 10-19; Sec. III B)                  */
/* ========================================================================== */

/* Band = first..last grid index where the reference amplitude is non-zero
   (h0 != 0, Sec. III B).  Edges: nbins+1 targets log-spaced from f(kmin) to
   f(kmax), rounded to the nearest grid index, endpoints exact, duplicates
   dropped.  Returns the number of bins (edges has that + 1 entries) or -1 when
   the band has fewer than two points. */
long oracle_het_edges_hm(const double* th0, double f0, double df, long n, double t_obs,
                         unsigned modes, int nbins, long* edges, long* band)
{
    w0_t w;
    w0_setup(th0, &w);
    long kmin = -1, kmax = -1;
    for (long k = 0; k < n; ++k) {
        double f = f0 + k * df;
        int on = 0;   /* some selected mode of h0 is non-zero at f */
        for (int b = 0; b < 6 && !on; ++b) {
            if (!(modes & (1u << b))) continue;
            double f2 = 2.0 * f / HM_M[b];
            on = w0_amp(&w, f2, w0_time(&w, f2), t_obs) != 0.0;
        }
        if (on) {
            if (kmin < 0) kmin = k;
            kmax = k;
        }
    }
    band[0] = kmin; band[1] = kmax;
    if (kmin < 0 || kmax <= kmin || nbins < 1) return -1;
    double flo = f0 + kmin * df, fhi = f0 + kmax * df;
    long m = 0;
    for (int b = 0; b <= nbins; ++b) {
        long k;
        if (b == 0) k = kmin;
        else if (b == nbins) k = kmax;
        else {
            double ft = flo * pow(fhi / flo, (double)b / nbins);
            k = llround((ft - f0) / df);
            if (k < kmin) k = kmin;
            if (k > kmax) k = kmax;
        }
        if (m == 0 || k > edges[m - 1]) edges[m++] = k;
    }
    return m - 1;
}

long oracle_het_edges(const double* th0, double f0, double df, long n, double t_obs, int nbins,
                      long* edges, long* band)
{
    return oracle_het_edges_hm(th0, f0, df, n, t_obs, 1u, nbins, edges, band);
}

/* Summary data for the reference th0 (Eqs. 15, 16, 18, 19), per bin b and channel c,
   sum[(b*3 + c)*6 + {0..5}] = Re A0, Im A0, Re A1, Im A1, B0, B1, with
   A0 = sum_{k in b} d conj(h0)/S df, A1 = sum d conj(h0)/S (f - f_b) df,
   B0 = sum |h0|^2/S df, B1 = sum |h0|^2/S (f - f_b) df, f_b = bin centre.
   Bin b holds k in [e_b, e_{b+1}), the last bin also holds e_E.
   h0e[(e*3 + c)] = h0 at edge e (complex interleaved).
   Returns the number of bins E (or -1); edges needs nbins+1 entries. */
long oracle_het_prepare_hm(const double* th0, double f0, double df, long n, double t_obs,
                           unsigned modes, const double* d, const double* S, int nbins,
                           long* edges, double* sum, double* h0e, double* dd_out)
{
    long band[2];
    long E = oracle_het_edges_hm(th0, f0, df, n, t_obs, modes, nbins, edges, band);
    *dd_out = oracle_inner(d, d, S, n, df, 0);
    if (E < 1) return -1;
    const cplx* cd = (const cplx*)d;
    long kmin = edges[0], kmax = edges[E];
    long nb = kmax - kmin + 1;
    double* f = malloc(sizeof(double) * nb);
    for (long i = 0; i < nb; ++i) f[i] = f0 + (kmin + i) * df;
    cplx* h0 = malloc(sizeof(cplx) * 3 * nb);
    template_eval_modes(th0, t_obs, f, nb, modes, h0, NULL);
    for (long b = 0; b < E; ++b) {
        long klo = edges[b], khi = edges[b + 1];
        long kend = (b == E - 1) ? khi + 1 : khi;
        double fb = 0.5 * ((f0 + klo * df) + (f0 + khi * df));
        for (int c = 0; c < 3; ++c) {
            cplx a0 = 0.0, a1 = 0.0;
            double b0 = 0.0, b1 = 0.0;
            for (long k = klo; k < kend; ++k) {
                double fk = f0 + k * df;
                cplx hk = h0[c * nb + (k - kmin)];
                double Sk = S[c * n + k];
                cplx dk = cd[c * n + k];
                a0 += dk * conj(hk) / Sk * df;
                a1 += dk * conj(hk) / Sk * (fk - fb) * df;
                b0 += creal(hk * conj(hk)) / Sk * df;
                b1 += creal(hk * conj(hk)) / Sk * (fk - fb) * df;
            }
            double* o = sum + (b * 3 + c) * 6;
            o[0] = creal(a0); o[1] = cimag(a0); o[2] = creal(a1); o[3] = cimag(a1);
            o[4] = b0; o[5] = b1;
        }
    }
    for (long e = 0; e <= E; ++e)
        for (int c = 0; c < 3; ++c) {
            cplx v = h0[c * nb + (edges[e] - kmin)];
            h0e[2 * (e * 3 + c)] = creal(v);
            h0e[2 * (e * 3 + c) + 1] = cimag(v);
        }
    free(h0);
    free(f);
    return E;
}

long oracle_het_prepare(const double* th0, double f0, double df, long n, double t_obs,
                        const double* d, const double* S, int nbins,
                        long* edges, double* sum, double* h0e, double* dd_out)
{
    return oracle_het_prepare_hm(th0, f0, df, n, t_obs, 1u, d, S, nbins, edges, sum, h0e, dd_out);
}

/* Contraction from template values at the edges (Eqs. 14 and 17): he is
   [W][E+1][3] complex.  r = h/h0 (0 where h0 = 0), r0 = (r_lo + r_hi)/2,
   r1 = (r_hi - r_lo)/(f_hi - f_lo);
   <d|h> ~ 4 Re sum_b sum_c A0 conj(r0) + A1 conj(r1),
   <h|h> ~ 4 sum_b sum_c B0 |r0|^2 + 2 B1 Re(r0 conj(r1)),
   out as in oracle_direct. */
void oracle_het_contract(long E, const long* edges, double f0, double df, const double* sum,
                         const double* h0e, double dd, const double* he, long W, double* out)
{
    const cplx* ch0 = (const cplx*)h0e;
    const cplx* che = (const cplx*)he;
    for (long i = 0; i < W; ++i) {
        const cplx* hw = che + i * (E + 1) * 3;
        double dh = 0.0, hh = 0.0;
        for (long b = 0; b < E; ++b) {
            double flo = f0 + edges[b] * df, fhi = f0 + edges[b + 1] * df;
            for (int c = 0; c < 3; ++c) {
                cplx h0lo = ch0[b * 3 + c], h0hi = ch0[(b + 1) * 3 + c];
                cplx rlo = h0lo != 0.0 ? hw[b * 3 + c] / h0lo : 0.0;
                cplx rhi = h0hi != 0.0 ? hw[(b + 1) * 3 + c] / h0hi : 0.0;
                cplx r0 = 0.5 * (rlo + rhi);
                cplx r1 = (rhi - rlo) / (fhi - flo);
                const double* s = sum + (b * 3 + c) * 6;
                cplx A0 = s[0] + I * s[1], A1 = s[2] + I * s[3];
                double B0 = s[4], B1 = s[5];
                dh += 4.0 * creal(A0 * conj(r0) + A1 * conj(r1));
                hh += 4.0 * (B0 * creal(r0 * conj(r0)) + 2.0 * B1 * creal(r0 * conj(r1)));
            }
        }
        out[i] = -0.5 * (dd + hh - 2.0 * dh);
        out[W + i] = dh;
        out[2 * W + i] = hh;
    }
}

/* Heterodyned likelihood of W walkers (SoA [11][W]) against a prepared reference, templates
   of the modes of the mask (the reference's). */
void oracle_het_loglike_hm(const double* th, long W, long E, const long* edges, double f0,
                           double df, double t_obs, unsigned modes, const double* sum,
                           const double* h0e, double dd, double* out)
{
    double* fe = malloc(sizeof(double) * (E + 1));
    for (long e = 0; e <= E; ++e) fe[e] = f0 + edges[e] * df;
    cplx* he = malloc(sizeof(cplx) * W * (E + 1) * 3);
#pragma omp parallel for schedule(dynamic)
    for (long i = 0; i < W; ++i) {
        double t[11];
        theta_col(th, W, i, t);
        cplx* tmp = malloc(sizeof(cplx) * 3 * (E + 1));
        template_eval_modes(t, t_obs, fe, E + 1, modes, tmp, NULL);
        for (long e = 0; e <= E; ++e)
            for (int c = 0; c < 3; ++c) he[(i * (E + 1) + e) * 3 + c] = tmp[c * (E + 1) + e];
        free(tmp);
    }
    oracle_het_contract(E, edges, f0, df, sum, h0e, dd, (const double*)he, W, out);
    free(he);
    free(fe);
}

void oracle_het_loglike(const double* th, long W, long E, const long* edges, double f0,
                        double df, double t_obs, const double* sum, const double* h0e,
                        double dd, double* out)
{
    oracle_het_loglike_hm(th, W, E, edges, f0, df, t_obs, 1u, sum, h0e, dd, out);
}

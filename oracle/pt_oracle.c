/*
 * FP64 CPU oracle of one iteration of the parallel-tempered ensemble sampler that
 * drives all three pipeline modules (Katz, arXiv:2111.01064, Sec. III, the paragraph
 * after Table I).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header or
 * constant generator with the CUDA library and never reads a value the CUDA
 * library produced.
 *
 * What it computes, in the order of the method:
 *   ensemble      T temperatures (inverse temperatures beta_t, target L^beta_t pi),
 *                 W walkers each; walker (t, k) is column t W + k of the state.
 *   coordinates   the sampler moves x = (ln M_T, q, a1, a2, D_L, phi_ref, cos iota,
 *                 lambda, sin beta, psi, t_ref); the prior of Table I is uniform in x
 *                 on a box [lo, hi] (log-uniform M_T, uniform cos iota and sin beta),
 *                 so ln pi is constant inside and -inf outside.
 *   half steps    the walkers of each temperature are split into halves
 *                 [0, W/2) and [W/2, W); the first half moves using the second as its
 *                 complementary ensemble, then the second using the updated first.
 *   proposals     with probability p_stretch the affine-invariant stretch move of
 *                 Goodman & Weare (2010): Y = x_j + z (x_k - x_j), x_j a uniformly
 *                 drawn walker of the complementary half, z from g(z) ~ 1/sqrt(z)
 *                 on [1/a, a], acceptance factor z^(d-1), d = 11.  Otherwise a
 *                 sky-mode hop (Sec. III): longitudinal modes shift lambda and psi
 *                 together by n pi/2 (n = 0..3; lambda taken mod 2 pi, psi mod pi);
 *                 the latitudinal mode flips sin beta, cos iota and cos psi
 *                 (psi -> pi - psi).  Three varieties: a mode drawn from all eight
 *                 (n uniform in 0..3, flip with probability 1/2), a longitudinal
 *                 change only (n uniform in 1..3), a latitudinal flip only.  The hops
 *                 are group actions drawn uniformly, hence symmetric proposals.
 *   acceptance    tempered Metropolis: accept iff Y is inside the prior box and
 *                 ln u < ln(factor) + beta_t (lnL(Y) - lnL(x_k)).
 *   swaps         parallel tempering between adjacent temperatures, hottest pair
 *                 first (Vousden, Farr & Mandel 2016): at level i (hot i, cold i-1)
 *                 cold walker k is paired with hot walker sigma_i(k), sigma_i a
 *                 random permutation, and the pair exchanges states iff
 *                 ln u < (beta_{i-1} - beta_i)(lnL_hot - lnL_cold).
 *   ladder        optionally adapted after every iteration (Vousden, Farr & Mandel 2016):
 *                 with T_t = 1/beta_t, S_t = ln(T_t - T_{t-1}) for the intermediate
 *                 temperatures 1 <= t <= T-2 moves by kappa(n) (A_t - A_{t+1}), A_t the
 *                 fraction of accepted swaps of pair (t, t-1) in this iteration and
 *                 kappa(n) = (1/nu) n0/(n + n0) at iteration n; the coldest and the hottest
 *                 temperatures stay fixed, the others are rebuilt from T_0 upwards.
 *   randomness    Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), key = the
 *                 64-bit seed, counter = (item, purpose, step low, step high); 53-bit
 *                 uniforms from two words; permutations by sorting 48-bit random
 *                 keys (ties broken by index).
 *
 * The likelihood is the oracle's heterodyned lnL (oracle_het_loglike, Sec. II B) at
 * theta(x), or, for the sampler's own pins, a diagonal Gaussian in x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_het_loglike(const double* th, long W, long E, const long* edges, double f0,
                        double df, double t_obs, const double* sum, const double* h0e,
                        double dd, double* out);
void oracle_direct_hm(const double* th, long W, double f0, double df, long n, double t_obs,
                      unsigned modes, const double* d, const double* S, double* out);

enum { NPAR = 11 };
enum { K_STRETCH = 0, K_SKY_ALL = 1, K_SKY_LON = 2, K_SKY_LAT = 3 };
enum { P_PROPOSE = 0x10, P_ACCEPT = 0x20, P_SWAP_KEY = 0x100, P_SWAP_ACC = 0x200 };

static const double PI_ = 3.141592653589793;
static const double HALF_PI_ = 1.5707963267948966;
static const double TWO_PI_ = 6.283185307179586;

/* ---- Philox4x32-10 ---------------------------------------------------------
   One round maps (c0, c1, c2, c3) with key (k0, k1) to
   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
   M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is advanced by the Weyl constants
   (0x9E3779B9, 0xBB67AE85) between rounds; ten rounds. */
void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    memcpy(out, c, sizeof c);
}

static void draw(uint64_t seed, uint32_t item, uint32_t purpose, uint64_t step, uint32_t* r)
{
    const uint32_t ctr[4] = {item, purpose, (uint32_t)step, (uint32_t)(step >> 32)};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, r);
}

/* uniform in [0, 1) with 53 random bits: (a >> 5) 2^26 + (b >> 6), times 2^-53 */
static double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* theta(x): M_T = exp(ln M_T), iota = acos(cos iota), beta = asin(sin beta) */
static void theta_of_x(const double* x, double* th)
{
    for (int p = 0; p < NPAR; ++p) th[p] = x[p];
    th[0] = exp(x[0]);
    th[6] = acos(x[6]);
    th[8] = asin(x[8]);
}

void oracle_pt_theta(const double* x, long n, double* th)
{
    for (long i = 0; i < n; ++i) {
        double a[NPAR], b[NPAR];
        for (int p = 0; p < NPAR; ++p) a[p] = x[p * n + i];
        theta_of_x(a, b);
        for (int p = 0; p < NPAR; ++p) th[p * n + i] = b[p];
    }
}

static double reduce_period(double v, double P)
{
    while (v >= P) v -= P;
    while (v < 0.0) v += P;
    return v;
}

static int in_box(const double* y, const double* lo, const double* hi)
{
    for (int p = 0; p < NPAR; ++p)
        if (!(y[p] >= lo[p] && y[p] <= hi[p])) return 0;
    return 1;
}

/* The random choices of one proposal: kind, complement walker (stretch), z, and the
   sky mode (n, m).  item = t (W/2) + k' for the k'-th moving walker of temperature t. */
typedef struct {
    int kind;
    long j;
    double z;
    int n, m;
} choice_t;

static choice_t choose(uint64_t seed, uint64_t step, int half, long item, long W,
                       const double* probs, double a)
{
    uint32_t r[4];
    draw(seed, (uint32_t)item, P_PROPOSE + (uint32_t)half, step, r);
    choice_t c = {0, -1, 1.0, 0, 0};
    const double u = (double)r[0] * (1.0 / 4294967296.0);
    const double c1 = probs[0], c2 = c1 + probs[1], c3 = c2 + probs[2];
    c.kind = u < c1 ? K_STRETCH : u < c2 ? K_SKY_ALL : u < c3 ? K_SKY_LON : K_SKY_LAT;
    const long Wh = W / 2;
    c.j = (1 - half) * Wh + (long)(((uint64_t)r[1] * (uint64_t)Wh) >> 32);
    const double s = (a - 1.0) * u53(r[2], r[3]) + 1.0;
    c.z = s * s / a;
    if (c.kind == K_SKY_ALL) {
        c.n = (int)(r[2] >> 30);
        c.m = (int)(r[3] >> 31);
    } else if (c.kind == K_SKY_LON) {
        c.n = 1 + (int)(((uint64_t)r[2] * 3u) >> 32);
    } else if (c.kind == K_SKY_LAT) {
        c.m = 1;
    }
    return c;
}

/* test access to the draws: out = (kind, j, z, n, m) */
void oracle_pt_choice(uint64_t seed, uint64_t step, int half, long item, long W,
                      const double* probs, double a, double* out)
{
    const choice_t c = choose(seed, step, half, item, W, probs, a);
    out[0] = c.kind;
    out[1] = (double)c.j;
    out[2] = c.z;
    out[3] = c.n;
    out[4] = c.m;
}

/* sky-mode map (n longitudinal quarter turns, m latitudinal flip) on x */
void oracle_pt_sky(double* x, int n, int m)
{
    x[7] = reduce_period(x[7] + (double)n * HALF_PI_, TWO_PI_);
    x[9] = reduce_period(x[9] + (double)n * HALF_PI_, PI_);
    if (m) {
        x[8] = -x[8];
        x[6] = -x[6];
        x[9] = PI_ - x[9];
    }
}

/* ---- likelihoods --------------------------------------------------------- */
typedef struct {
    int kind; /* 0 heterodyne, 1 diagonal Gaussian in x, 2 direct */
    long E;
    const long* edges;
    double f0, df, t_obs;
    const double *sum, *h0e;
    double dd;
    const double *mu, *sigma;
    long n;                    /* direct: grid size, data d [3][n] complex, PSD S [3][n] */
    const double *d, *S;
    unsigned modes;            /* direct: harmonic mode mask of the templates */
} like_t;

/* out[3][n] (lnL, <d|h>, <h|h>) for n points x[11][n] */
static void loglike(const like_t* L, const double* x, long n, double* out)
{
    if (L->kind == 0 || L->kind == 2) {
        double* th = malloc(sizeof(double) * NPAR * n);
        oracle_pt_theta(x, n, th);
        if (L->kind == 0)
            oracle_het_loglike(th, n, L->E, L->edges, L->f0, L->df, L->t_obs, L->sum, L->h0e,
                               L->dd, out);
        else
            oracle_direct_hm(th, n, L->f0, L->df, L->n, L->t_obs, L->modes, L->d, L->S, out);
        free(th);
        return;
    }
    for (long i = 0; i < n; ++i) {
        double s = 0.0;
        for (int p = 0; p < NPAR; ++p)
            if (L->sigma[p] > 0.0) {
                const double r = (x[p * n + i] - L->mu[p]) / L->sigma[p];
                s += r * r;
            }
        out[i] = -0.5 * s;
        out[n + i] = 0.0;
        out[2 * n + i] = 0.0;
    }
}

static int cmp_u64(const void* a, const void* b)
{
    const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : x > y;
}

/* ---- one iteration ----------------------------------------------------------
   x: [11][T W], out: [3][T W] (lnL, <d|h>, <h|h> of the current states), updated in
   place.  counters (int64, 10 T): [0, 4T) proposals per (t, kind), [4T, 8T) accepted
   per (t, kind), [8T, 9T) accepted swaps per level i (pair i, i-1; entry 0 unused),
   [9T, 10T) proposed swaps per level. */
static void adapt_ladder(double* betas, long T, const long* acc_now, long W, uint64_t step, double nu,
                         double n0)
{
    if (T < 3) return;
    const double kappa = (1.0 / nu) * n0 / ((double)step + n0);
    double* Tt = malloc(sizeof(double) * T);
    double* S = malloc(sizeof(double) * T);
    for (long t = 0; t < T; ++t) Tt[t] = 1.0 / betas[t];
    for (long t = 1; t <= T - 2; ++t) {
        const double A = (double)acc_now[t] / (double)W, A1 = (double)acc_now[t + 1] / (double)W;
        S[t] = log(Tt[t] - Tt[t - 1]) + kappa * (A - A1);
    }
    for (long t = 1; t <= T - 2; ++t) {
        Tt[t] = Tt[t - 1] + exp(S[t]);
        betas[t] = 1.0 / Tt[t];
    }
    free(S);
    free(Tt);
}

static void iteration(double* x, double* out, long T, long W, double* betas,
                      const double* lo, const double* hi, const double* probs, double a,
                      uint64_t seed, uint64_t step, const like_t* L, long* counters,
                      double adapt_nu, double adapt_n0)
{
    const long N = T * W, Wh = W / 2, M = T * Wh;
    double* y = malloc(sizeof(double) * NPAR * M);
    double* fac = malloc(sizeof(double) * M);
    int* ok = malloc(sizeof(int) * M);
    int* kind = malloc(sizeof(int) * M);
    double* oy = malloc(sizeof(double) * 3 * M);
    for (int half = 0; half < 2; ++half) {
        /* proposals of every moving walker from the current state */
        for (long t = 0; t < T; ++t)
            for (long kp = 0; kp < Wh; ++kp) {
                const long item = t * Wh + kp, k = half * Wh + kp;
                const long col = t * W + k;
                const choice_t c = choose(seed, step, half, item, W, probs, a);
                double v[NPAR];
                for (int p = 0; p < NPAR; ++p) v[p] = x[p * N + col];
                if (c.kind == K_STRETCH) {
                    const long colj = t * W + c.j;
                    for (int p = 0; p < NPAR; ++p) {
                        const double xj = x[p * N + colj];
                        v[p] = xj + c.z * (v[p] - xj);
                    }
                    fac[item] = (double)(NPAR - 1) * log(c.z);
                } else {
                    oracle_pt_sky(v, c.n, c.m);
                    fac[item] = 0.0;
                }
                ok[item] = in_box(v, lo, hi);
                kind[item] = c.kind;
                for (int p = 0; p < NPAR; ++p) y[p * M + item] = v[p];
            }
        loglike(L, y, M, oy);
        for (long t = 0; t < T; ++t)
            for (long kp = 0; kp < Wh; ++kp) {
                const long item = t * Wh + kp, col = t * W + half * Wh + kp;
                uint32_t r[4];
                draw(seed, (uint32_t)item, P_ACCEPT + (uint32_t)half, step, r);
                const double lnu = log(u53(r[0], r[1]));
                const double la = fac[item] + betas[t] * (oy[item] - out[col]);
                const int acc = ok[item] && lnu < la;
                counters[t * 4 + kind[item]] += 1;
                if (acc) {
                    counters[4 * T + t * 4 + kind[item]] += 1;
                    for (int p = 0; p < NPAR; ++p) x[p * N + col] = y[p * M + item];
                    for (int q = 0; q < 3; ++q) out[q * N + col] = oy[q * M + item];
                }
            }
    }
    /* temperature swaps, hottest pair first */
    uint64_t* keys = malloc(sizeof(uint64_t) * W);
    long* acc_now = calloc((size_t)T, sizeof(long));
    for (long i = T - 1; i >= 1; --i) {
        for (long k = 0; k < W; ++k) {
            uint32_t r[4];
            draw(seed, (uint32_t)k, P_SWAP_KEY + (uint32_t)i, step, r);
            keys[k] = ((uint64_t)r[0] << 32) | ((uint64_t)(r[1] & 0xFFFF0000u)) | (uint64_t)k;
        }
        qsort(keys, (size_t)W, sizeof(uint64_t), cmp_u64);
        for (long k = 0; k < W; ++k) {
            const long hot = i * W + (long)(keys[k] & 0xFFFFu), cold = (i - 1) * W + k;
            uint32_t r[4];
            draw(seed, (uint32_t)k, P_SWAP_ACC + (uint32_t)i, step, r);
            const double lnu = log(u53(r[0], r[1]));
            const double la = (betas[i - 1] - betas[i]) * (out[hot] - out[cold]);
            counters[9 * T + i] += 1;
            if (lnu < la) {
                counters[8 * T + i] += 1;
                acc_now[i] += 1;
                for (int p = 0; p < NPAR; ++p) {
                    const double s = x[p * N + hot];
                    x[p * N + hot] = x[p * N + cold];
                    x[p * N + cold] = s;
                }
                for (int q = 0; q < 3; ++q) {
                    const double s = out[q * N + hot];
                    out[q * N + hot] = out[q * N + cold];
                    out[q * N + cold] = s;
                }
            }
        }
    }
    if (adapt_nu > 0.0) adapt_ladder(betas, T, acc_now, W, step, adapt_nu, adapt_n0);
    free(acc_now);
    free(keys);
    free(oy);
    free(kind);
    free(ok);
    free(fac);
    free(y);
}

/* n_iter iterations from step step0 with the heterodyned likelihood. */
/* betas (in/out): the ladder, adapted in place when adapt_nu > 0 (adapt_n0 the lag). */
void oracle_pt_run_het(double* x, double* out, long T, long W, double* betas,
                       const double* lo, const double* hi, const double* probs, double a,
                       uint64_t seed, uint64_t step0, long n_iter, long E, const long* edges,
                       double f0, double df, double t_obs, const double* sum, const double* h0e,
                       double dd, long* counters, double adapt_nu, double adapt_n0)
{
    like_t L = {0, E, edges, f0, df, t_obs, sum, h0e, dd, NULL, NULL, 0, NULL, NULL, 1u};
    for (long s = 0; s < n_iter; ++s)
        iteration(x, out, T, W, betas, lo, hi, probs, a, seed, step0 + (uint64_t)s, &L, counters,
                  adapt_nu, adapt_n0);
}

/* n_iter iterations with the direct likelihood (Module 1 of Sec. III) on the grid
   f_k = f0 + k df, k < n, data d [3][n] complex and PSD S [3][n], templates of the
   harmonic modes of the mask (the higher-mode posterior of Sec. III C uses this form). */
void oracle_pt_run_direct(double* x, double* out, long T, long W, double* betas,
                          const double* lo, const double* hi, const double* probs, double a,
                          uint64_t seed, uint64_t step0, long n_iter, double f0, double df,
                          long n, double t_obs, unsigned modes, const double* d, const double* S,
                          long* counters)
{
    like_t L = {2, 0, NULL, f0, df, t_obs, NULL, NULL, 0, NULL, NULL, n, d, S, modes};
    for (long s = 0; s < n_iter; ++s)
        iteration(x, out, T, W, betas, lo, hi, probs, a, seed, step0 + (uint64_t)s, &L, counters,
                  0.0, 0.0);
}

/* The same sampler on lnL = -1/2 sum_p ((x_p - mu_p)/sigma_p)^2 (sigma_p = 0: x_p
   unconstrained); the chain of every sample is appended to trace[n_iter][T][11]
   (the state after each iteration, for moment checks). */
void oracle_pt_run_gauss(double* x, double* out, long T, long W, double* betas,
                         const double* lo, const double* hi, const double* probs, double a,
                         uint64_t seed, uint64_t step0, long n_iter, const double* mu,
                         const double* sigma, long* counters, double* trace, double adapt_nu,
                         double adapt_n0, double* beta_trace)
{
    like_t L = {1, 0, NULL, 0, 0, 0, NULL, NULL, 0, mu, sigma, 0, NULL, NULL, 1u};
    const long N = T * W;
    for (long s = 0; s < n_iter; ++s) {
        iteration(x, out, T, W, betas, lo, hi, probs, a, seed, step0 + (uint64_t)s, &L, counters,
                  adapt_nu, adapt_n0);
        if (beta_trace) memcpy(beta_trace + s * T, betas, sizeof(double) * T);
        if (trace) memcpy(trace + s * NPAR * N, x, sizeof(double) * NPAR * N);
    }
}

/* lnL of the Gaussian target at x[11][n] (the tests score initial states with it) */
void oracle_pt_gauss_loglike(const double* x, long n, const double* mu, const double* sigma,
                             double* out)
{
    like_t L = {1, 0, NULL, 0, 0, 0, NULL, NULL, 0, mu, sigma, 0, NULL, NULL, 1u};
    loglike(&L, x, n, out);
}

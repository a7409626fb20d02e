// Device arithmetic of the parallel-tempered sampler (Katz, arXiv:2111.01064, Sec. III): the
// ensemble state, Philox4x32-10 draws, the coordinates x -> theta and one walker's proposal
// and acceptance test.  Shared by the sampler's own kernels and by the heterodyne kernel's
// fused variant, which proposes in its walker setup and accepts in its epilogue.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mbh {
namespace pt {

constexpr int kPar = 11;
constexpr int kMaxTemps = 64;
constexpr int kMaxWalkers = 8192;   // per temperature (16-bit walker index in the swap keys)

enum { K_STRETCH = 0, K_SKY_ALL = 1, K_SKY_LON = 2, K_SKY_LAT = 3 };
enum : uint32_t { P_PROPOSE = 0x10, P_ACCEPT = 0x20, P_SWAP_KEY = 0x100, P_SWAP_ACC = 0x200 };

constexpr double kPtPi = 3.141592653589793;
constexpr double kPtHalfPi = 1.5707963267948966;
constexpr double kPtTwoPi = 6.283185307179586;

// Several independent ensembles (one per source, or independent chains of one source) step
// together: ensemble e owns slots [e T W, (e+1) T W) and half-step items [e M, (e+1) M),
// M = T W/2, and draws its random numbers with the key seed_e = seed + e 0x9E3779B97F4A7C15,
// so each ensemble is exactly a single-ensemble sampler with seed seed_e.
struct PtArgs {
    double* x;              // [11][N] positions, physical columns (N = n_ens T W)
    double* out;            // [3][N] lnL, <d|h>, <h|h>
    int32_t* map;           // [N] slot -> column
    double* y;              // [11][M] proposals of the moving half
    double* theta;          // [11][N] likelihood input (first M columns during a half step)
    double* out_p;          // [3][M] likelihood of the proposals
    double* fac;            // [M] log acceptance factor (d-1) ln z of stretch moves
    int32_t* flag;          // [M] inside-prior bit | kind << 1
    int32_t* perm;          // [T][W] hot partner of cold walker k at level i
    double* lnu_acc;        // [2][n_ens M] ln u of the acceptance tests of both half steps
    double* lnu_swap;       // [n_ens][T][W] ln u of the swap tests (level 0 unused)
    double* betas;          // [n_ens][T] (adapted in place when adapt_nu > 0)
    unsigned long long* counters;   // [n_ens][10 T]
    unsigned int* done;     // swap-kernel blocks finished in this iteration (last one advances step)
    unsigned long long* step;       // iteration counter
    double lo[kPar], hi[kPar];
    double c1, c2, c3;      // cumulative proposal probabilities
    double a, am1;          // stretch scale and a - 1
    double adapt_nu, adapt_n0;   // ladder adaptation (nu > 0 enables)
    uint64_t seed;
    int32_t T, W, n_ens;
};

__device__ __forceinline__ uint64_t ens_seed(const PtArgs& A, int e)
{
    return A.seed + (uint64_t)e * 0x9E3779B97F4A7C15ull;
}

// ---- Philox4x32-10 -------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t item, uint32_t purpose, uint64_t step)
{
    return philox(item, purpose, (uint32_t)step, (uint32_t)(step >> 32), (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

// 53-bit uniform in [0, 1); every operation is exact
__device__ __forceinline__ double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

// v mod P for v in [-2P, 4P) (a coordinate of the prior box plus at most 3 quarter turns);
// the bounded loops leave values outside that range outside [0, P), i.e. outside the prior.
__device__ __forceinline__ double reduce_period(double v, double P)
{
    for (int i = 0; i < 4 && v >= P; ++i) v = __dsub_rn(v, P);
    for (int i = 0; i < 2 && v < 0.0; ++i) v = __dadd_rn(v, P);
    return v;
}

__device__ __forceinline__ void theta_of_x(const double (&x)[kPar], double (&th)[kPar])
{
#pragma unroll
    for (int p = 0; p < kPar; ++p) th[p] = x[p];
    th[0] = exp(fmin(x[0], 700.0));
    th[6] = acos(fmin(fmax(x[6], -1.0), 1.0));   // clamps act only outside the prior box
    th[8] = asin(fmin(fmax(x[8], -1.0), 1.0));
}

// Proposal of moving walker `item` (= e M + t W/2 + k') of half `half`: Y (v), theta(Y) or
// theta of the current point when Y leaves the prior box (th), the log acceptance factor and the
// flag (inside-prior bit | kind << 1).  Explicitly rounded float64, so Y is reproducible bit for
// bit.  The ensemble's own walkers and draws only: ensembles are independent.
__device__ __forceinline__ void propose_item(const PtArgs& A, int half, int32_t item, uint64_t step,
                                             double (&v)[kPar], double (&th)[kPar], double& fac,
                                             int32_t& flag)
{
    const int32_t Wh = A.W / 2, M = A.T * Wh;
    const int64_t N = (int64_t)A.n_ens * A.T * A.W;
    const int32_t e = item / M, li = item - e * M;
    const int32_t base = e * A.T * A.W;
    const int32_t t = li / Wh, kp = li - t * Wh;
    const int32_t col = A.map[base + t * A.W + half * Wh + kp];
    const uint4 r = draw(ens_seed(A, e), (uint32_t)li, P_PROPOSE + (uint32_t)half, step);
    const double u = (double)r.x * (1.0 / 4294967296.0);
    const int kind = u < A.c1 ? K_STRETCH : u < A.c2 ? K_SKY_ALL : u < A.c3 ? K_SKY_LON : K_SKY_LAT;
    double xk[kPar];
#pragma unroll
    for (int p = 0; p < kPar; ++p) xk[p] = v[p] = A.x[(int64_t)p * N + col];
    fac = 0.0;
    if (kind == K_STRETCH) {
        const int32_t j = (1 - half) * Wh + (int32_t)(((uint64_t)r.y * (uint64_t)Wh) >> 32);
        const int32_t colj = A.map[base + t * A.W + j];
        const double s = __dadd_rn(__dmul_rn(A.am1, u53(r.z, r.w)), 1.0);
        const double z = __ddiv_rn(__dmul_rn(s, s), A.a);
#pragma unroll
        for (int p = 0; p < kPar; ++p) {
            const double xj = A.x[(int64_t)p * N + colj];
            v[p] = __dadd_rn(xj, __dmul_rn(z, __dsub_rn(v[p], xj)));
        }
        fac = (double)(kPar - 1) * log(z);
    } else {
        int n = 0, m = 0;
        if (kind == K_SKY_ALL) {
            n = (int)(r.z >> 30);
            m = (int)(r.w >> 31);
        } else if (kind == K_SKY_LON) {
            n = 1 + (int)(((uint64_t)r.z * 3u) >> 32);
        } else {
            m = 1;
        }
        const double shift = __dmul_rn((double)n, kPtHalfPi);
        v[7] = reduce_period(__dadd_rn(v[7], shift), kPtTwoPi);
        v[9] = reduce_period(__dadd_rn(v[9], shift), kPtPi);
        if (m) {
            v[8] = -v[8];
            v[6] = -v[6];
            v[9] = __dsub_rn(kPtPi, v[9]);
        }
    }
    bool ok = true;
#pragma unroll
    for (int p = 0; p < kPar; ++p) ok = ok && (v[p] >= A.lo[p] && v[p] <= A.hi[p]);
    theta_of_x(ok ? v : xk, th);   // outside the prior: score the current point (rejected anyway)
    flag = (ok ? 1 : 0) | (kind << 1);
}

// Tempered Metropolis test of moving walker `item` with proposal lnL lnl_p; returns the
// decision (the column, and the ensemble's counter offset plus temperature, come back for the
// update: counters of (e, t) start at e 10 T, the temperature index is t).
__device__ __forceinline__ bool accept_test(const PtArgs& A, int half, int32_t item, double lnl_p, double fac,
                                            int32_t flag, int32_t& col, int& t, int& cbase)
{
    const int32_t Wh = A.W / 2, M = A.T * Wh;
    const int32_t e = item / M, li = item - e * M;
    t = li / Wh;
    const int32_t kp = li - t * Wh;
    col = A.map[e * A.T * A.W + t * A.W + half * Wh + kp];
    cbase = e * 10 * A.T;
    const double dl = __dsub_rn(lnl_p, A.out[col]);
    const double la = __dadd_rn(fac, __dmul_rn(A.betas[e * A.T + t], dl));
    return (flag & 1) && A.lnu_acc[(int64_t)half * A.n_ens * M + item] < la;
}

}  // namespace pt
}  // namespace mbh

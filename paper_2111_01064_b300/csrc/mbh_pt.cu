// Parallel-tempered ensemble sampler iteration on the device (Katz, arXiv:2111.01064, Sec. III,
// the sampler shared by all pipeline modules): stretch moves (Goodman & Weare 2010) for most
// proposals, sky-mode hops (the eight LISA-frame sky modes of Sec. III, three varieties),
// tempered Metropolis acceptance against L^beta pi, and swaps between adjacent temperatures,
// hottest pair first (Vousden, Farr & Mandel 2016).  The likelihood of every proposal batch is
// the library's heterodyned (Sec. II B) or direct (Sec. II) likelihood.
//
// One iteration = 9 launches, no host synchronisation, captured once in a CUDA graph:
//   pt_draws_kernel    ln u of every acceptance and swap test (state-independent)
//   pt_perm_kernel     random permutations of every swap level (state-independent; one block
//                      per level, bitonic sort of 48-bit Philox keys in shared memory); both
//                      on a side stream forked at the start of the iteration, joined before the
//                      first acceptance and before the swaps, so they overlap the half steps
//   for each half h:   pt_propose_kernel -> likelihood of the T*W/2 proposals -> pt_accept_kernel
//   pt_swap_kernel     the swap levels in order, hottest first (one block per ensemble; the two
//                      temperatures of a level are held in shared memory, or every temperature
//                      when T W (8 + 4) bytes fit: pt_swap_resident_kernel), then the step
//                      counter advances.
//
// Layout: positions x[11][N] and (lnL, <d|h>, <h|h>) out[3][N] stay in physical columns; a map
// slot -> column (slot = t W + k, walker k of temperature t) makes a swap an exchange of two
// map entries instead of 2 x 14 doubles.  Walkers are read and written through the map.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), key = seed, counter =
// (item, purpose, step low, step high), so every draw is fixed by (seed, step, purpose, item)
// and independent of launch configuration.  The proposal arithmetic uses explicitly rounded
// float64 operations (no contraction), so positions are reproducible bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mbh_df.cuh"
#include "mbh_internal.cuh"
#include "mbh_pt.cuh"

using namespace mbh;

namespace {

using namespace mbh::pt;
constexpr int kThreads = 256;      // rescoring and gathers
constexpr int kStepThreads = 32;   // propose/accept: 8192 walkers -> 256 blocks over all SMs
constexpr int kSortThreads = 1024;
// shared memory of pt_swap_resident_kernel: all T x W lnL and map entries (8 x 2048 walkers
// need 192 KiB), leaving room for the static arrays under the 227 KiB limit
constexpr size_t kSwapResidentBytes = 200 * 1024;

// ---- kernels -------------------------------------------------------------------------------
__global__ void __launch_bounds__(kStepThreads) pt_propose_kernel(const PtArgs A, int half)
{
    const int32_t M = A.n_ens * A.T * (A.W / 2);   // moving walkers of all ensembles
    const int32_t item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= M) return;
    double v[kPar], th[kPar], fac;
    int32_t flag;
    propose_item(A, half, item, *A.step, v, th, fac, flag);
#pragma unroll
    for (int p = 0; p < kPar; ++p) {
        A.y[(int64_t)p * M + item] = v[p];
        A.theta[(int64_t)p * M + item] = th[p];
    }
    A.fac[item] = fac;
    A.flag[item] = flag;
}

__global__ void __launch_bounds__(kStepThreads) pt_accept_kernel(const PtArgs A, int half)
{
    const int32_t M = A.n_ens * A.T * (A.W / 2);
    const int64_t N = (int64_t)A.n_ens * A.T * A.W;
    const int32_t item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= M) return;
    int32_t col;
    int t, cb;
    const int32_t f = A.flag[item];
    const int kind = f >> 1;
    const bool acc = accept_test(A, half, item, A.out_p[item], A.fac[item], f, col, t, cb);
    // counters of ensemble e at cb: [0, 4T) proposals per (t, kind), [4T, 8T) accepted
    atomicAdd(&A.counters[cb + t * 4 + kind], 1ull);
    if (acc) {
        atomicAdd(&A.counters[cb + 4 * A.T + t * 4 + kind], 1ull);
#pragma unroll
        for (int p = 0; p < kPar; ++p) A.x[(int64_t)p * N + col] = A.y[(int64_t)p * M + item];
#pragma unroll
        for (int q = 0; q < 3; ++q) A.out[(int64_t)q * N + col] = A.out_p[(int64_t)q * M + item];
    }
}

// ln u of every acceptance and swap test of the iteration (state-independent, float64 log on
// the whole GPU): items [0, 2 Mt) acceptance tests of half 0 and 1 (Mt = n_ens M), then
// n_ens (T-1) W swap tests.
__global__ void __launch_bounds__(kThreads) pt_draws_kernel(const PtArgs A)
{
    const int32_t M = A.T * (A.W / 2), Mt = A.n_ens * M;
    const int64_t per = (int64_t)(A.T - 1) * A.W;
    const int64_t n = 2 * (int64_t)Mt + (int64_t)A.n_ens * per;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint64_t step = *A.step;
    if (q < 2 * (int64_t)Mt) {
        const int half = (int)(q / Mt);
        const int32_t item = (int32_t)(q - (int64_t)half * Mt);
        const int32_t e = item / M, li = item - e * M;
        const uint4 r = draw(ens_seed(A, e), (uint32_t)li, P_ACCEPT + (uint32_t)half, step);
        A.lnu_acc[q] = log(u53(r.x, r.y));
    } else {
        const int64_t s = q - 2 * (int64_t)Mt;
        const int e = (int)(s / per);
        const int64_t r0 = s - (int64_t)e * per;
        const int i = 1 + (int)(r0 / A.W);
        const int32_t k = (int32_t)(r0 - (int64_t)(i - 1) * A.W);
        const uint4 r = draw(ens_seed(A, e), (uint32_t)k, P_SWAP_ACC + (uint32_t)i, step);
        A.lnu_swap[((int64_t)e * A.T + i) * A.W + k] = log(u53(r.x, r.y));
    }
}

// One block per (ensemble e, swap level i): sort the keys (48 random bits, then the walker
// index) of the hot temperature's walkers; perm[e][i][k] = hot partner of cold walker k.
__global__ void __launch_bounds__(kSortThreads) pt_perm_kernel(const PtArgs A, int Wp)
{
    extern __shared__ unsigned long long keys[];
    const int e = blockIdx.x / (A.T - 1), i = blockIdx.x % (A.T - 1) + 1;
    const uint64_t step = *A.step;
    for (int k = threadIdx.x; k < Wp; k += blockDim.x) {
        if (k < A.W) {
            const uint4 r = draw(ens_seed(A, e), (uint32_t)k, P_SWAP_KEY + (uint32_t)i, step);
            keys[k] = ((unsigned long long)r.x << 32) | (unsigned long long)(r.y & 0xFFFF0000u) |
                      (unsigned long long)k;
        } else {
            keys[k] = ~0ull;
        }
    }
    __syncthreads();
    for (int size = 2; size <= Wp; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int q = threadIdx.x; q < Wp / 2; q += blockDim.x) {
                const int lo = 2 * q - (q & (stride - 1)), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = keys[lo], b = keys[hi];
                if ((a > b) == up) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
    for (int k = threadIdx.x; k < A.W; k += blockDim.x)
        A.perm[((int64_t)e * A.T + i) * A.W + k] = (int32_t)(keys[k] & 0xFFFFull);
}

// The swap test cu < db (lh - lc) exactly as float64 decides it, without float64 instructions
// in all but ~1e-7 of the cases (one SM's float64 pipe would otherwise bound the swap levels):
// the operands as float pairs (integer splitting, 2^-48 relative), the difference and the
// product in float32 with a bound on their error, float64 only inside that bound.
__device__ __forceinline__ bool swap_test(double cu, double db, float dbf, double lh, double lc)
{
    const auto finite_small = [](double x) {   // |x| < 2^100 (and finite): the split is exact enough
        return ((unsigned long long)__double_as_longlong(x) >> 52 & 0x7ffull) < 1023ull + 100ull;
    };
    if (finite_small(lh) && finite_small(lc) && finite_small(cu)) {
        const f2 a = split_f64(lh, 0), b = split_f64(lc, 0), u = split_f64(cu, 0);
        const float d = (a.hi - b.hi) + (a.lo - b.lo);
        const float la = dbf * d, uf = u.hi + u.lo;
        // float32 rounding of the difference, product and ln u (a few 1e-7 relative), the pairs'
        // 2^-48 and the pair-split of db, with a factor ~4 of margin
        const float err = 2e-6f * (fabsf(la) + fabsf(uf)) + 1e-13f * dbf * (fabsf(a.hi) + fabsf(b.hi)) + 1e-37f;
        if (uf < la - err) return true;
        if (uf > la + err) return false;
    }
    return cu < __dmul_rn(db, __dsub_rn(lh, lc));
}

// After the swap levels (thread 0 of an ensemble's block): ladder adaptation from this
// iteration's swap acceptances, then the last ensemble block to finish advances the step.
__device__ void swap_epilogue(const PtArgs& A, double* betas, const unsigned int* acc_now, uint64_t step)
{
    const int T = A.T, W = A.W;
    // ladder adaptation (Vousden, Farr & Mandel 2016): S_t = ln(T_t - T_{t-1}) moves by
    // kappa (A_t - A_{t+1}), kappa = (1/nu) n0/(n + n0); coldest and hottest fixed
    if (A.adapt_nu > 0.0 && T >= 3) {
        const double kappa = __ddiv_rn(__dmul_rn(__ddiv_rn(1.0, A.adapt_nu), A.adapt_n0),
                                       __dadd_rn((double)step, A.adapt_n0));
        double Tt[kMaxTemps], S[kMaxTemps];
        for (int t = 0; t < T; ++t) Tt[t] = __ddiv_rn(1.0, betas[t]);
        for (int t = 1; t <= T - 2; ++t) {
            const double a0 = __ddiv_rn((double)acc_now[t], (double)W);
            const double a1 = __ddiv_rn((double)acc_now[t + 1], (double)W);
            S[t] = __dadd_rn(log(__dsub_rn(Tt[t], Tt[t - 1])), __dmul_rn(kappa, __dsub_rn(a0, a1)));
        }
        for (int t = 1; t <= T - 2; ++t) {
            Tt[t] = __dadd_rn(Tt[t - 1], exp(S[t]));
            betas[t] = __ddiv_rn(1.0, Tt[t]);
        }
    }
    // the last ensemble block to finish advances the step: every block has read it by then
    __threadfence();
    if (atomicAdd(A.done, 1u) == (unsigned int)(A.n_ens - 1)) {
        *A.done = 0u;
        *A.step = step + 1;
    }
}

// Swap levels in order, hottest first; the hot and cold temperatures of a level are held in
// shared memory (lnL and map entries).  Thread t handles walkers k = t + j blockDim (j < J);
// while level i is decided, the next level's inputs (the colder temperature's map entries and
// then their lnL, the permutation, ln u) are already being loaded into registers, so each
// level costs its arithmetic and barriers rather than two dependent global round trips.
// Thread 0 advances the step counter at the end.
template <int J>
__global__ void __launch_bounds__(kSortThreads) pt_swap_kernel(const PtArgs A)
{
    extern __shared__ double sm[];
    const int W = A.W, T = A.T;
    const int e = blockIdx.x;                               // one block per ensemble
    int32_t* map = A.map + (int64_t)e * T * W;
    const int32_t* perm = A.perm + (int64_t)e * T * W;
    const double* lnu_swap = A.lnu_swap + (int64_t)e * T * W;
    double* betas = A.betas + (int64_t)e * T;
    unsigned long long* counters = A.counters + (int64_t)e * 10 * T;
    double* lnl = sm;                                       // [2][W]
    int32_t* mp = reinterpret_cast<int32_t*>(sm + 2 * W);   // [2][W]
    __shared__ unsigned int acc_level;
    __shared__ unsigned int acc_now[kMaxTemps];
    const uint64_t step = *A.step;
    if (T > 1) {
        int32_t pm[J], pp[J];
        double pl[J], pu[J];
        // level i's inputs: map and lnL of temperature i-1, permutation and ln u of level i
        auto issue = [&](int i) {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int k = threadIdx.x + j * blockDim.x;
                if (k < W) {
                    pm[j] = map[(i - 1) * W + k];
                    pp[j] = perm[(int64_t)i * W + k];
                    pu[j] = lnu_swap[(int64_t)i * W + k];
                }
            }
        };
        auto gather = [&]() {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int k = threadIdx.x + j * blockDim.x;
                if (k < W) pl[j] = A.out[pm[j]];
            }
        };
        int hot = 0;
        for (int k = threadIdx.x; k < W; k += blockDim.x) {
            const int32_t c = map[(T - 1) * W + k];
            mp[k] = c;
            lnl[k] = A.out[c];
        }
        issue(T - 1);
        gather();
        for (int i = T - 1; i >= 1; --i) {
            const int cold = hot ^ 1;
            int32_t cp[J];
            double cu[J];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int k = threadIdx.x + j * blockDim.x;
                if (k < W) {
                    mp[cold * W + k] = pm[j];
                    lnl[cold * W + k] = pl[j];
                    cp[j] = pp[j];
                    cu[j] = pu[j];
                }
            }
            if (threadIdx.x == 0) acc_level = 0;
            __syncthreads();
            if (i > 1) issue(i - 1);   // in flight while this level is decided
            const double db = __dsub_rn(betas[i - 1], betas[i]);
            const float dbf = (float)db;
            unsigned int mine = 0;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int k = threadIdx.x + j * blockDim.x;
                if (k >= W) continue;
                const int h = cp[j];
                if (swap_test(cu[j], db, dbf, lnl[hot * W + h], lnl[cold * W + k])) {
                    const double l = lnl[hot * W + h];
                    lnl[hot * W + h] = lnl[cold * W + k];
                    lnl[cold * W + k] = l;
                    const int32_t c = mp[hot * W + h];
                    mp[hot * W + h] = mp[cold * W + k];
                    mp[cold * W + k] = c;
                    ++mine;
                }
            }
            if (i > 1) gather();
            if (mine) atomicAdd(&acc_level, mine);
            __syncthreads();
            for (int k = threadIdx.x; k < W; k += blockDim.x) map[i * W + k] = mp[hot * W + k];
            if (threadIdx.x == 0) {
                counters[8 * T + i] += acc_level;
                counters[9 * T + i] += (unsigned long long)W;
                acc_now[i] = acc_level;
            }
            __syncthreads();
            hot = cold;
        }
        for (int k = threadIdx.x; k < W; k += blockDim.x) map[k] = mp[hot * W + k];
    }
    __syncthreads();
    if (threadIdx.x == 0) swap_epilogue(A, betas, acc_now, step);
}

// The same swap levels with every temperature's lnL and map entries resident in shared memory
// (T W (8 + 4) bytes, when that fits): the state is read once at the start and written back
// once at the end, each level is decided from shared memory with one barrier, and the next
// level's permutation and ln u (independent of the state) load while the current level is
// decided.  Decisions, order and counters are those of pt_swap_kernel.
template <int J>
__global__ void __launch_bounds__(kSortThreads) pt_swap_resident_kernel(const PtArgs A)
{
    extern __shared__ double sm[];
    const int W = A.W, T = A.T;
    const int e = blockIdx.x;                               // one block per ensemble
    const int TW = T * W;
    int32_t* map = A.map + (int64_t)e * TW;
    const int32_t* perm = A.perm + (int64_t)e * TW;
    const double* lnu_swap = A.lnu_swap + (int64_t)e * TW;
    double* betas = A.betas + (int64_t)e * T;
    unsigned long long* counters = A.counters + (int64_t)e * 10 * T;
    double* lnl = sm;                                       // [T][W]
    int32_t* mp = reinterpret_cast<int32_t*>(sm + TW);      // [T][W]
    __shared__ unsigned int acc_now[kMaxTemps];
    __shared__ double bs[kMaxTemps];
    const uint64_t step = *A.step;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        acc_now[t] = 0;
        bs[t] = betas[t];
    }
    // map first (independent loads), then the lnL behind each entry (eight in flight a thread)
#pragma unroll 8
    for (int s = threadIdx.x; s < TW; s += blockDim.x) mp[s] = map[s];
#pragma unroll 8
    for (int s = threadIdx.x; s < TW; s += blockDim.x) lnl[s] = A.out[mp[s]];
    if (T > 1) {
        int32_t cp[J], np[J];
        double cu[J], nu[J];
        auto load = [&](int i, int32_t (&p)[J], double (&u)[J]) {
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int k = threadIdx.x + j * blockDim.x;
                if (k < W) {
                    p[j] = perm[(int64_t)i * W + k];
                    u[j] = lnu_swap[(int64_t)i * W + k];
                }
            }
        };
        load(T - 1, cp, cu);
        __syncthreads();
        for (int i = T - 1; i >= 1; --i) {
            if (i > 1) load(i - 1, np, nu);   // in flight while this level is decided
            const double db = __dsub_rn(bs[i - 1], bs[i]);
            const float dbf = (float)db;
            double* lh = lnl + i * W;
            double* lc = lnl + (i - 1) * W;
            int32_t* mh = mp + i * W;
            int32_t* mc = mp + (i - 1) * W;
            unsigned int mine = 0;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int k = threadIdx.x + j * blockDim.x;
                if (k >= W) continue;
                const int h = cp[j];
                if (swap_test(cu[j], db, dbf, lh[h], lc[k])) {
                    const double l = lh[h];
                    lh[h] = lc[k];
                    lc[k] = l;
                    const int32_t c = mh[h];
                    mh[h] = mc[k];
                    mc[k] = c;
                    ++mine;
                }
            }
            if (mine) atomicAdd(&acc_now[i], mine);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < J; ++j) {
                cp[j] = np[j];
                cu[j] = nu[j];
            }
        }
    }
    for (int s = threadIdx.x; s < TW; s += blockDim.x) map[s] = mp[s];
    for (int t = 1 + (int)threadIdx.x; t < T; t += blockDim.x) {
        counters[8 * T + t] += acc_now[t];
        counters[9 * T + t] += (unsigned long long)W;
    }
    __syncthreads();
    if (threadIdx.x == 0) swap_epilogue(A, betas, acc_now, step);
}

// theta(x) of every physical column (rescoring)
__global__ void pt_theta_kernel(const double* __restrict__ x, int64_t N, double* __restrict__ th)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    double v[kPar], t[kPar];
#pragma unroll
    for (int p = 0; p < kPar; ++p) v[p] = x[p * N + c];
    theta_of_x(v, t);
#pragma unroll
    for (int p = 0; p < kPar; ++p) th[p * N + c] = t[p];
}

// slot-ordered copy of the state; or, with scatter != 0, load positions in slot order
__global__ void pt_gather_kernel(const PtArgs A, const double* __restrict__ xs, double* __restrict__ xo,
                                 double* __restrict__ oo, int scatter)
{
    const int64_t N = (int64_t)A.n_ens * A.T * A.W;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    if (scatter) {
        A.map[s] = (int32_t)s;
#pragma unroll
        for (int p = 0; p < kPar; ++p) A.x[p * N + s] = xs[p * N + s];
        return;
    }
    const int32_t c = A.map[s];
    if (xo)
#pragma unroll
        for (int p = 0; p < kPar; ++p) xo[p * N + s] = A.x[p * N + c];
    if (oo)
#pragma unroll
        for (int q = 0; q < 3; ++q) oo[q * N + s] = A.out[q * N + c];
}

// best (largest lnL, lowest slot on ties) walker of temperature t of ensemble e -> res[14]
__global__ void __launch_bounds__(kSortThreads) pt_best_kernel(const PtArgs A, int e, int t, double* res)
{
    __shared__ double bv[32];
    __shared__ int bs[32];
    const int64_t N = (int64_t)A.n_ens * A.T * A.W;
    const int32_t* map = A.map + (int64_t)e * A.T * A.W;
    double best = -INFINITY;
    int slot = -1;
    for (int k = threadIdx.x; k < A.W; k += blockDim.x) {
        const double v = A.out[map[t * A.W + k]];
        if (slot < 0 || v > best) {
            best = v;
            slot = k;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int os = __shfl_down_sync(0xffffffffu, slot, o);
        if (os >= 0 && (slot < 0 || ov > best || (ov == best && os < slot))) {
            best = ov;
            slot = os;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        bv[warp] = best;
        bs[warp] = slot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            if (bs[w] >= 0 && (slot < 0 || bv[w] > best || (bv[w] == best && bs[w] < slot))) {
                best = bv[w];
                slot = bs[w];
            }
        const int32_t c = map[t * A.W + (slot < 0 ? 0 : slot)];
        for (int p = 0; p < kPar; ++p) res[p] = A.x[p * N + c];
        for (int q = 0; q < 3; ++q) res[kPar + q] = A.out[q * N + c];
    }
}

}  // namespace

struct mbh_pt {
    int device = -1;
    PtArgs A{};
    mbh_precision precision = MBH_MIXED;
    std::vector<const mbh_ref*> refs;   // one per ensemble (heterodyned likelihood)
    const mbh_data* data = nullptr;      // or the data of the direct likelihood
    mbh_het_config cfg{8, 0, 0};
    uint32_t modes = 1u;     // direct likelihood: harmonic modes of the templates
    bool fused = false;      // half steps as one fused heterodyne launch each
    bool fuse_ok = false;    // the caller allows fusion (mixed precision, not opted out)
    PtArgs* A_dev = nullptr; // device copy of A for the fused kernel
    int Wp = 0;
    double* res = nullptr;   // device [14] for mbh_pt_best
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t side = nullptr;   // permutation sorts, concurrent with the half steps
    cudaEvent_t fork = nullptr, join = nullptr, join_draws = nullptr;
};

namespace {

void free_pt(mbh_pt* P)
{
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->side) {
        cudaStreamSynchronize(P->side);
        cudaStreamDestroy(P->side);
    }
    if (P->fork) cudaEventDestroy(P->fork);
    if (P->join) cudaEventDestroy(P->join);
    if (P->join_draws) cudaEventDestroy(P->join_draws);
    PtArgs& A = P->A;
    void* bufs[] = {A.x, A.out, A.map, A.y, A.theta, A.out_p, A.fac, A.flag, A.perm, A.lnu_acc, A.lnu_swap,
                    A.betas, A.counters, A.step, A.done, P->res, P->A_dev};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete P;
}

// likelihood of the first n columns of A.theta into dst [3][n]; the columns are n/n_ens per
// ensemble, in ensemble order
mbh_status likelihood(mbh_pt* P, int64_t n, double* dst, cudaStream_t st)
{
    if (!P->refs.empty()) {
        const int ne = (int)P->refs.size();
        std::vector<int64_t> off(ne + 1);
        for (int e = 0; e <= ne; ++e) off[e] = n / ne * e;
        return het_loglike_batch_cfg(P->refs.data(), off.data(), ne, P->A.theta, P->precision, &P->cfg, dst, st);
    }
    return direct_loglike_batch_hm(P->data, P->A.theta, n, P->modes, P->precision, dst, st);
}

mbh_status rescore(mbh_pt* P, cudaStream_t st)
{
    const int64_t N = (int64_t)P->A.n_ens * P->A.T * P->A.W;
    pt_theta_kernel<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, st>>>(P->A.x, N, P->A.theta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pt_theta_kernel");
    return likelihood(P, N, P->A.out, st);
}

mbh_status queue_iteration(mbh_pt* P, cudaStream_t st)
{
    const PtArgs& A = P->A;
    const int32_t M = A.n_ens * A.T * (A.W / 2);   // moving walkers of all ensembles
    const unsigned gM = (unsigned)((M + kStepThreads - 1) / kStepThreads);
    cudaError_t e = cudaSuccess;
    // state-independent work on a side stream while the first half step runs: ln u of every
    // test of the iteration, then the permutations of the swap levels
    e = cudaEventRecord(P->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->side, P->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "fork");
    const int64_t nd = 2 * (int64_t)M + (int64_t)A.n_ens * (A.T - 1) * A.W;
    pt_draws_kernel<<<(unsigned)((nd + kThreads - 1) / kThreads), kThreads, 0, P->side>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pt_draws_kernel");
    if ((e = cudaEventRecord(P->join_draws, P->side)) != cudaSuccess) return cuda_fail(e, "join");
    if (A.T > 1) {
        pt_perm_kernel<<<A.n_ens * (A.T - 1), kSortThreads, sizeof(unsigned long long) * P->Wp, P->side>>>(A, P->Wp);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pt_perm_kernel");
    }
    if ((e = cudaEventRecord(P->join, P->side)) != cudaSuccess) return cuda_fail(e, "join");
    for (int half = 0; half < 2; ++half) {
        if (P->fused) {   // proposal, likelihood and acceptance in one launch
            if (half == 0 && (e = cudaStreamWaitEvent(st, P->join_draws, 0)) != cudaSuccess)
                return cuda_fail(e, "join");
            if (mbh_status s = het_launch_fused_pt(P->refs.data(), (int)P->refs.size(), M / A.n_ens, P->cfg, P->precision,
                                                   P->A_dev, half, st))
                return s;
            continue;
        }
        pt_propose_kernel<<<gM, kStepThreads, 0, st>>>(A, half);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pt_propose_kernel");
        if (mbh_status s = likelihood(P, M, A.out_p, st)) return s;
        if (half == 0 && (e = cudaStreamWaitEvent(st, P->join_draws, 0)) != cudaSuccess)
            return cuda_fail(e, "join");
        pt_accept_kernel<<<gM, kStepThreads, 0, st>>>(A, half);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pt_accept_kernel");
    }
    if ((e = cudaStreamWaitEvent(st, P->join, 0)) != cudaSuccess) return cuda_fail(e, "join");
    const size_t swap_smem = (sizeof(double) + sizeof(int32_t)) * 2 * A.W;
    const size_t resident_smem = (sizeof(double) + sizeof(int32_t)) * (size_t)A.T * A.W;
    const int J = (A.W + kSortThreads - 1) / kSortThreads;
    const unsigned ne = (unsigned)A.n_ens;   // one block per ensemble
    if (resident_smem <= kSwapResidentBytes && J <= 2) {
        if (J <= 1) pt_swap_resident_kernel<1><<<ne, kSortThreads, resident_smem, st>>>(A);
        else pt_swap_resident_kernel<2><<<ne, kSortThreads, resident_smem, st>>>(A);
    } else if (J <= 1) pt_swap_kernel<1><<<ne, kSortThreads, swap_smem, st>>>(A);
    else if (J <= 2) pt_swap_kernel<2><<<ne, kSortThreads, swap_smem, st>>>(A);
    else if (J <= 4) pt_swap_kernel<4><<<ne, kSortThreads, swap_smem, st>>>(A);
    else pt_swap_kernel<8><<<ne, kSortThreads, swap_smem, st>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "pt_swap_kernel");
    return MBH_OK;
}

void drop_graph(mbh_pt* P)
{
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    P->exec = nullptr;
    P->graph = nullptr;
}

mbh_status build_graph(mbh_pt* P)
{
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "graph stream");
    mbh_status status = MBH_OK;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        status = queue_iteration(P, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (status == MBH_OK && e2 != cudaSuccess) status = cuda_fail(e2, "graph capture");
        if (status == MBH_OK) {
            e2 = cudaGraphInstantiate(&P->exec, g, 0);
            if (e2 != cudaSuccess) status = cuda_fail(e2, "graph instantiate");
            P->graph = g;
        } else if (g) {
            cudaGraphDestroy(g);
        }
    } else {
        status = cuda_fail(e, "begin capture");
    }
    cudaStreamDestroy(cs);
    if (status != MBH_OK) drop_graph(P);
    return status;
}

}  // namespace

extern "C" mbh_status mbh_pt_create_multi(const mbh_pt_opts* o, const mbh_ref* const* refs, int32_t n_ens,
                                          const mbh_data* data, const double* betas_host, const double* x_dev,
                                          void* stream, mbh_pt** out)
{
    if (!out) return fail(MBH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!o || !betas_host || !x_dev) return fail(MBH_EINVAL, "NULL opts/betas/x");
    if ((refs == nullptr) == (data == nullptr)) return fail(MBH_EINVAL, "give exactly one of refs and data");
    if (n_ens < 1 || n_ens > 1024) return fail(MBH_EINVAL, "n_ens %d not in [1, 1024]", n_ens);
    if (refs)
        for (int32_t e = 0; e < n_ens; ++e)
            if (!refs[e]) return fail(MBH_EINVAL, "refs[%d] is NULL", e);
    if (o->ntemps < 1 || o->ntemps > kMaxTemps) return fail(MBH_EINVAL, "ntemps %d not in [1, %d]", o->ntemps, kMaxTemps);
    if (o->walkers < 4 || o->walkers > kMaxWalkers || (o->walkers & 1))
        return fail(MBH_EINVAL, "walkers %d: even, in [4, %d]", o->walkers, kMaxWalkers);
    if (!(o->a > 1.0)) return fail(MBH_EINVAL, "stretch scale a must be > 1");
    double csum = 0.0;
    for (int i = 0; i < 4; ++i) {
        if (!(o->probs[i] >= 0.0)) return fail(MBH_EINVAL, "negative proposal probability");
        csum += o->probs[i];
    }
    if (!(csum > 0.0 && csum <= 1.0 + 1e-12)) return fail(MBH_EINVAL, "proposal probabilities must sum to (0, 1]");
    for (int p = 0; p < kPar; ++p)
        if (!(o->lo[p] <= o->hi[p])) return fail(MBH_EINVAL, "prior box: lo[%d] > hi[%d]", p, p);
    if (o->adapt_time > 0.0 && !(o->adapt_lag > 0.0)) return fail(MBH_EINVAL, "adapt_lag must be > 0");
    if ((int64_t)n_ens * o->ntemps * o->walkers > 0x3fffffff) return fail(MBH_EINVAL, "ensemble too large");
    for (int64_t t = 0; t < (int64_t)n_ens * o->ntemps; ++t)
        if (!(betas_host[t] >= 0.0) || !std::isfinite(betas_host[t])) return fail(MBH_EINVAL, "betas must be finite and >= 0");
    if (o->precision != MBH_FP64 && o->precision != MBH_MIXED && o->precision != MBH_MIXED_F32)
        return fail(MBH_EINVAL, "unknown precision");
    const uint32_t modes = o->modes ? o->modes : 1u;
    if (data)
        if (mbh_status s = check_modes(modes, o->precision == MBH_MIXED_F32 ? MBH_MIXED : o->precision)) return s;
    if (mbh_status s = check_device()) return s;
    int dev = -1;
    cudaGetDevice(&dev);
    bool all22 = true;
    if (refs)
        for (int32_t e = 0; e < n_ens; ++e) {
            if (refs[e]->device != dev) return fail(MBH_EINVAL, "refs[%d] lives on another device", e);
            all22 = all22 && refs[e]->modes == 1u;
        }
    if (data && data->device != dev) return fail(MBH_EINVAL, "data lives on another device");

    mbh_pt* P = new (std::nothrow) mbh_pt;
    if (!P) return fail(MBH_ENOMEM, "host allocation");
    P->device = dev;
    if (refs) P->refs.assign(refs, refs + n_ens);
    P->data = data;
    P->precision = o->precision;
    P->modes = modes;
    if (o->het_config.threads_per_walker) P->cfg = o->het_config;
    PtArgs& A = P->A;
    A.T = o->ntemps;
    A.W = o->walkers;
    A.n_ens = n_ens;
    A.seed = o->seed;
    A.a = o->a;
    A.am1 = o->a - 1.0;
    A.adapt_nu = o->adapt_time > 0.0 ? o->adapt_time : 0.0;
    A.adapt_n0 = o->adapt_lag;
    A.c1 = o->probs[0];
    A.c2 = A.c1 + o->probs[1];
    A.c3 = A.c2 + o->probs[2];
    std::memcpy(A.lo, o->lo, sizeof A.lo);
    std::memcpy(A.hi, o->hi, sizeof A.hi);
    P->Wp = 1;
    while (P->Wp < A.W) P->Wp <<= 1;
    const int64_t N = (int64_t)n_ens * A.T * A.W, M = N / 2;
    // default launch shape of the mixed-precision half steps: enough threads per walker for
    // about one wave of the register-capped 224-thread blocks (28 warps per SM): 16 threads per
    // walker up to 12288 moving walkers, 8 above (threads per walker fixes the summation order,
    // so a sampler keeps the one it was created with)
    if (!o->het_config.threads_per_walker && P->precision == MBH_MIXED_F32) P->cfg.threads_per_walker = M <= 12288 ? 16 : 8;
    // MBH_MIXED: the extended-precision kernel; half steps of at most 12288 walkers fill the
    // GPU better with 8 threads per walker (8192 walkers: 0.260 ms against 0.292 ms with 4)
    if (!o->het_config.threads_per_walker && P->precision == MBH_MIXED) P->cfg.threads_per_walker = M <= 12288 ? 8 : 4;
    const int64_t NT = (int64_t)n_ens * A.T;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void**)&A.x, sizeof(double) * kPar * N);
    alloc((void**)&A.out, sizeof(double) * 3 * N);
    alloc((void**)&A.map, sizeof(int32_t) * N);
    alloc((void**)&A.y, sizeof(double) * kPar * M);
    alloc((void**)&A.theta, sizeof(double) * kPar * N);
    alloc((void**)&A.out_p, sizeof(double) * 3 * M);
    alloc((void**)&A.fac, sizeof(double) * M);
    alloc((void**)&A.flag, sizeof(int32_t) * M);
    alloc((void**)&A.perm, sizeof(int32_t) * N);
    alloc((void**)&A.lnu_acc, sizeof(double) * 2 * M);
    alloc((void**)&A.lnu_swap, sizeof(double) * N);
    alloc((void**)&A.betas, sizeof(double) * NT);
    alloc((void**)&A.counters, sizeof(unsigned long long) * 10 * NT);
    alloc((void**)&A.step, sizeof(unsigned long long));
    alloc((void**)&A.done, sizeof(unsigned int));
    alloc((void**)&P->res, sizeof(double) * 14);
    alloc((void**)&P->A_dev, sizeof(PtArgs));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join_draws, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_pt(P);
        return e == cudaErrorMemoryAllocation ? fail(MBH_ENOMEM, "sampler buffers") : cuda_fail(e, "sampler buffers");
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pt_perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(unsigned long long) * kMaxWalkers));
    const int swap_max = (int)((sizeof(double) + sizeof(int32_t)) * 2 * kMaxWalkers);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pt_swap_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, swap_max);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pt_swap_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, swap_max);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pt_swap_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, swap_max);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(pt_swap_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, swap_max);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pt_swap_resident_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSwapResidentBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pt_swap_resident_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSwapResidentBytes);
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned long long zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(A.betas, betas_host, sizeof(double) * NT, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.counters, 0, sizeof(unsigned long long) * 10 * NT, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(A.step, &zero, sizeof zero, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.done, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.perm, 0, sizeof(int32_t) * N, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->A_dev, &A, sizeof(PtArgs), cudaMemcpyHostToDevice, st);
    // fused half steps: the float32-ratio kernel (MBH_MIXED_F32) or the extended kernel
    // (MBH_MIXED), where a kernel exists for the launch shape
    {
        const int G = P->cfg.threads_per_walker;
        const int blk = P->cfg.block ? P->cfg.block : fused_pt_block(o->precision, G, M);
        const bool shape = o->precision == MBH_MIXED ? het_kernel_x_pt(G, blk).launch != nullptr
                                                     : het_kernel_mixed_pt(G, blk).launch != nullptr;
        P->fuse_ok = (o->precision == MBH_MIXED_F32 || o->precision == MBH_MIXED) && !o->no_fuse && shape;
    }
    P->fused = P->fuse_ok && refs != nullptr && all22;
    if (e != cudaSuccess) {
        free_pt(P);
        return cuda_fail(e, "sampler setup");
    }
    pt_gather_kernel<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, st>>>(A, x_dev, nullptr, nullptr, 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        free_pt(P);
        return cuda_fail(e, "pt_gather_kernel");
    }
    if (mbh_status s = rescore(P, st)) {
        free_pt(P);
        return s;
    }
    // the host-to-device copies above read host memory that the caller may release on return
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_pt(P);
        return cuda_fail(e, "sampler setup");
    }
    *out = P;
    return MBH_OK;
}

extern "C" mbh_status mbh_pt_create(const mbh_pt_opts* o, const mbh_ref* ref, const mbh_data* data,
                                    const double* betas_host, const double* x_dev, void* stream,
                                    mbh_pt** out)
{
    return mbh_pt_create_multi(o, ref ? &ref : nullptr, 1, data, betas_host, x_dev, stream, out);
}

extern "C" mbh_status mbh_pt_run(mbh_pt* P, int64_t n_iter, int32_t use_graph, void* stream)
{
    if (!P) return fail(MBH_EINVAL, "sampler is NULL");
    if (n_iter < 0) return fail(MBH_EINVAL, "n_iter < 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (use_graph && !P->exec)
        if (mbh_status s = build_graph(P)) return s;
    for (int64_t i = 0; i < n_iter; ++i) {
        if (use_graph) {
            cudaError_t e = cudaGraphLaunch(P->exec, st);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        } else if (mbh_status s = queue_iteration(P, st)) {
            return s;
        }
    }
    return MBH_OK;
}

extern "C" mbh_status mbh_pt_state(const mbh_pt* P, double* x_dev, double* out_dev, void* stream)
{
    if (!P) return fail(MBH_EINVAL, "sampler is NULL");
    const int64_t N = (int64_t)P->A.n_ens * P->A.T * P->A.W;
    pt_gather_kernel<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, (cudaStream_t)stream>>>(
        P->A, nullptr, x_dev, out_dev, 0);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "pt_gather_kernel");
}

extern "C" mbh_status mbh_pt_set_state(mbh_pt* P, const double* x_dev, void* stream)
{
    if (!P || !x_dev) return fail(MBH_EINVAL, "NULL sampler/x");
    const int64_t N = (int64_t)P->A.n_ens * P->A.T * P->A.W;
    cudaStream_t st = (cudaStream_t)stream;
    pt_gather_kernel<<<(unsigned)((N + kThreads - 1) / kThreads), kThreads, 0, st>>>(P->A, x_dev, nullptr, nullptr, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pt_gather_kernel");
    return rescore(P, st);
}

extern "C" mbh_status mbh_pt_set_ref_at(mbh_pt* P, int32_t ensemble, const mbh_ref* ref, void* stream)
{
    if (!P || !ref) return fail(MBH_EINVAL, "NULL sampler/ref");
    if (P->refs.empty()) return fail(MBH_EINVAL, "sampler uses the direct likelihood");
    if (ensemble < 0 || ensemble >= (int32_t)P->refs.size()) return fail(MBH_EINVAL, "ensemble %d out of range", ensemble);
    if (ref->device != P->device) return fail(MBH_EINVAL, "ref lives on another device");
    P->refs[ensemble] = ref;
    bool all22 = true;
    for (const mbh_ref* r : P->refs) all22 = all22 && r->modes == 1u;
    P->fused = P->fuse_ok && all22;
    drop_graph(P);   // the reference's tables are baked into the captured launches
    return rescore(P, (cudaStream_t)stream);
}

extern "C" mbh_status mbh_pt_set_ref(mbh_pt* P, const mbh_ref* ref, void* stream)
{
    if (P && P->A.n_ens != 1) return fail(MBH_EINVAL, "several ensembles: use mbh_pt_set_ref_at");
    return mbh_pt_set_ref_at(P, 0, ref, stream);
}

extern "C" mbh_status mbh_pt_set_betas(mbh_pt* P, const double* betas_host, void* stream)
{
    if (!P || !betas_host) return fail(MBH_EINVAL, "NULL sampler/betas");
    const int64_t NT = (int64_t)P->A.n_ens * P->A.T;
    for (int64_t t = 0; t < NT; ++t)
        if (!(betas_host[t] >= 0.0) || !std::isfinite(betas_host[t])) return fail(MBH_EINVAL, "betas must be finite and >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(P->A.betas, betas_host, sizeof(double) * NT,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "set betas");
}

extern "C" mbh_status mbh_pt_get_betas(const mbh_pt* P, double* betas_host, void* stream)
{
    if (!P || !betas_host) return fail(MBH_EINVAL, "NULL sampler/betas");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(betas_host, P->A.betas, sizeof(double) * P->A.n_ens * P->A.T,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "get betas");
}

extern "C" mbh_status mbh_pt_counters(const mbh_pt* P, int64_t* counters_host, uint64_t* step_host,
                                      void* stream)
{
    if (!P) return fail(MBH_EINVAL, "sampler is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (counters_host)
        e = cudaMemcpyAsync(counters_host, P->A.counters, sizeof(int64_t) * 10 * P->A.n_ens * P->A.T,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && step_host)
        e = cudaMemcpyAsync(step_host, P->A.step, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "read counters");
}

extern "C" mbh_status mbh_pt_best_at(const mbh_pt* P, int32_t ensemble, int32_t temp, double* x_host,
                                     double* out_host, void* stream)
{
    if (!P) return fail(MBH_EINVAL, "sampler is NULL");
    if (temp < 0 || temp >= P->A.T) return fail(MBH_EINVAL, "temperature %d out of range", temp);
    if (ensemble < 0 || ensemble >= P->A.n_ens) return fail(MBH_EINVAL, "ensemble %d out of range", ensemble);
    cudaStream_t st = (cudaStream_t)stream;
    pt_best_kernel<<<1, kSortThreads, 0, st>>>(P->A, ensemble, temp, P->res);
    cudaError_t e = cudaGetLastError();
    double r[14];
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, P->res, sizeof r, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "pt_best");
    if (x_host) std::memcpy(x_host, r, sizeof(double) * kPar);
    if (out_host) std::memcpy(out_host, r + kPar, sizeof(double) * 3);
    return MBH_OK;
}

extern "C" mbh_status mbh_pt_best(const mbh_pt* P, int32_t temp, double* x_host, double* out_host,
                                  void* stream)
{
    return mbh_pt_best_at(P, 0, temp, x_host, out_host, stream);
}

extern "C" void mbh_pt_free(mbh_pt* P)
{
    if (P) free_pt(P);
}

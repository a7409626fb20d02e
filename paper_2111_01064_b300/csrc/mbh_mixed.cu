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
#include "mbh_mixed.cuh"
#include "mbh_pt.cuh"

using namespace mbh;


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
    if (kind < 0 || kind > 6) return fail(MBH_EINVAL, "kind must be 0..6");
    if (n < 0) return fail(MBH_EINVAL, "n < 0");
    if (n == 0) return MBH_OK;
    if (!x_dev || !o1_dev || ((kind == 0 || kind == 5) && !o2_dev) || ((kind == 2 || kind == 4 || kind == 6) && !y_dev))
        return fail(MBH_EINVAL, "NULL buffer");
    if (mbh_status s = check_device()) return s;
    if (kind >= 5) return selftest_df(kind, x_dev, y_dev, n, o1_dev, o2_dev, (cudaStream_t)stream);
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
// O(1) (float32 range); per-point products are float32, sums float64.  Three blocks per SM
// (80 registers, 52.5 KB of shared memory each; a few bytes of spills in the set-up): 5 %
// faster than two (108 registers), the six-mode pass 7 %; four (64 registers) spill in the
// point loop and run slower.
constexpr int kDirFlush = 16;   // points per float32 partial sum in the fused mixed pass

template <int T, bool kHM>
__global__ void __launch_bounds__(kDirThreadsM, 3)
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
    direct_chunks(data->grid.n, tiles, 1 << 14, chunk, nchunks, 2);   // as the double-float pass
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
            if (active && e <= E) edge_delta_mixed_hm(wsd[lw], wsf[lw], wsh[lw], S.mix, e, modes, tob, dl);
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

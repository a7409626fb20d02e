// libmbhlike: CUDA kernels and C-ABI entry points for the batched LISA MBHB likelihood
// (Katz, arXiv:2111.01064, Sec. II).  Declarations and conventions: include/mbhlike.h.
//
// Kernels (all float64 here; the mixed-precision variants live in mbh_mixed.cu):
//   psd_kernel          analytic A/E/T PSD (Sec. II, remark under Eq. 3)
//   noise_kernel        Gaussian noise from standard normals (Sec. II)
//   template_kernel     W0 + R0 on the grid (Eqs. 7-9)
//   data_kernel         4 df d/S, 4 df/S and per-block <d|d> partials (Eq. 3)
//   direct_fused        template generation fused with the reduction (Eqs. 2-3, 7-9)
//   band_kernel         support of the reference template (Sec. III B: h0 != 0)
//   prep_items_kernel   per-(bin, sub-range) partial summary data (Eqs. 15-16, 18-19)
//   het_f64_kernel      heterodyned lnL, G threads per walker (Eqs. 14, 17)
// Every reduction is fixed-order (per-thread sequential, then a shuffle/shared-memory tree,
// then a sequential pass over block partials), so a result does not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mbhlike.h"
#include "mbh_df.cuh"
#include "mbh_internal.cuh"
#include "mbh_model.cuh"

using namespace mbh;

// ------------------------------------------------------------------------------------------
// error state
// ------------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

namespace mbh {
mbh_status fail(mbh_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

mbh_status cuda_fail(cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(MBH_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(MBH_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

mbh_status check_grid(const mbh_grid* g)
{
    if (!g) return fail(MBH_EINVAL, "grid is NULL");
    if (!(g->f0 > 0.0) || !(g->df > 0.0) || g->n < 2 || !(g->t_obs > 0.0) ||
        !std::isfinite(g->f0 + g->df * (double)g->n))
        return fail(MBH_EINVAL, "bad grid (f0=%g df=%g n=%lld t_obs=%g)", g->f0, g->df,
                    (long long)g->n, g->t_obs);
    return MBH_OK;
}

mbh_status check_device()
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n < 1) {
        cudaGetLastError();
        return fail(MBH_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    return MBH_OK;
}
}  // namespace mbh

extern "C" const char* mbh_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------------------------------
// PSD and noise
// ------------------------------------------------------------------------------------------
// x = 2 pi f L/c; S_acc = a^2 (1 + (4e-4/f)^2)(1 + (f/8e-3)^4)/(2 pi f c)^2,
// S_oms = o^2 (1 + (2e-3/f)^4)(2 pi f/c)^2;
// S_A = S_E = 8 sin^2 x [2 S_acc (3 + 2 cos x + cos 2x) + S_oms (2 + cos x)],
// S_T = 32 sin^2 x sin^2(x/2) [4 S_acc sin^2(x/2) + S_oms].
__global__ void psd_kernel(double f0, double df, int64_t n, double* __restrict__ S)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double f = f0 + (double)k * df;
        const double x = kTwoPi * f * kArmSec;
        const double r1 = 4e-4 / f, r2 = f / 8e-3, r3 = 2e-3 / f;
        const double wa = kTwoPi * f * kClight, wo = kTwoPi * f / kClight;
        const double sacc = 9e-30 * (1.0 + r1 * r1) * (1.0 + r2 * r2 * r2 * r2) / (wa * wa);
        const double soms = 2.25e-22 * (1.0 + r3 * r3 * r3 * r3) * (wo * wo);
        double sx, cx, sh, ch;
        sincos(x, &sx, &cx);
        sincos(0.5 * x, &sh, &ch);
        const double c2x = cx * cx - sx * sx;
        const double sa = 8.0 * sx * sx * (2.0 * sacc * (3.0 + 2.0 * cx + c2x) + soms * (2.0 + cx));
        const double st = 32.0 * sx * sx * sh * sh * (4.0 * sacc * sh * sh + soms);
        S[k] = sa;
        S[n + k] = sa;
        S[2 * n + k] = st;
    }
}

__global__ void noise_kernel(double df, int64_t n, const double* __restrict__ z,
                             const double* __restrict__ S, int accumulate,
                             double2* __restrict__ out)
{
    const int64_t m = 3 * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double sig = sqrt(S[i] / (4.0 * df));
        double2 v = {sig * z[2 * i], sig * z[2 * i + 1]};
        if (accumulate) {
            double2 o = out[i];
            v.x += o.x;
            v.y += o.y;
        }
        out[i] = v;
    }
}

static int grid_blocks(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 64));
}

extern "C" mbh_status mbh_psd_aet(const mbh_grid* grid, double* psd_dev, void* stream)
{
    if (mbh_status s = check_grid(grid)) return s;
    if (!psd_dev) return fail(MBH_EINVAL, "psd_dev is NULL");
    if (mbh_status s = check_device()) return s;
    psd_kernel<<<grid_blocks(grid->n, 256), 256, 0, (cudaStream_t)stream>>>(grid->f0, grid->df,
                                                                          grid->n, psd_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "mbh_psd_aet");
}

extern "C" mbh_status mbh_noise_aet(const mbh_grid* grid, const double* z_dev, const double* psd_dev,
                                    int32_t accumulate, void* noise_dev, void* stream)
{
    if (mbh_status s = check_grid(grid)) return s;
    if (!z_dev || !psd_dev || !noise_dev) return fail(MBH_EINVAL, "NULL buffer");
    if (mbh_status s = check_device()) return s;
    noise_kernel<<<grid_blocks(3 * grid->n, 256), 256, 0, (cudaStream_t)stream>>>(
        grid->df, grid->n, z_dev, psd_dev, accumulate, (double2*)noise_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "mbh_noise_aet");
}

// ------------------------------------------------------------------------------------------
// templates on the grid
// ------------------------------------------------------------------------------------------
constexpr int kTplThreads = 128;
constexpr int kTplPerThread = 4;

// block (chunk, walker): thread 0 derives the walker constants; every thread evaluates
// kTplPerThread grid points, coalesced per channel.
__global__ void __launch_bounds__(kTplThreads)
    template_f64_kernel(const double* __restrict__ theta, int64_t W, double f0, double df,
                        int64_t n, double t_obs, uint32_t modes, double2* __restrict__ h)
{
    __shared__ Walker ws;
    for (int64_t wi = blockIdx.y; wi < W; wi += gridDim.y) {
        __syncthreads();
        if (threadIdx.x == 0) walker_setup(theta, W, wi, ws, modes);
        __syncthreads();
        const int64_t base = (int64_t)blockIdx.x * kTplThreads * kTplPerThread + threadIdx.x;
#pragma unroll
        for (int j = 0; j < kTplPerThread; ++j) {
            const int64_t k = base + (int64_t)j * kTplThreads;
            if (k < n) {
                cd v[3];
                point_model_f64(ws, f0 + (double)k * df, t_obs, v);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    h[((int64_t)wi * 3 + c) * n + k] = make_double2(v[c].re, v[c].im);
            }
        }
    }
}

namespace mbh {
mbh_status launch_template_f64(const mbh_grid* g, const double* theta, int64_t W, double2* h,
                               cudaStream_t st, uint32_t modes = 1u)
{
    const int64_t per_block = (int64_t)kTplThreads * kTplPerThread;
    dim3 grid((unsigned)((g->n + per_block - 1) / per_block), (unsigned)std::min<int64_t>(W, 65535));
    template_f64_kernel<<<grid, kTplThreads, 0, st>>>(theta, W, g->f0, g->df, g->n, g->t_obs, modes, h);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "template kernel");
}
}  // namespace mbh

extern "C" mbh_status template_batch(const mbh_grid* grid, const double* theta_dev, int64_t W,
                                     mbh_precision precision, void* h_out_dev, void* stream)
{
    if (mbh_status s = check_grid(grid)) return s;
    if (W < 0) return fail(MBH_EINVAL, "W < 0");
    if (W == 0) return MBH_OK;
    if (!theta_dev || !h_out_dev) return fail(MBH_EINVAL, "NULL buffer");
    if (mbh_status s = check_device()) return s;
    if (precision == MBH_FP64)
        return launch_template_f64(grid, theta_dev, W, (double2*)h_out_dev, (cudaStream_t)stream);
    if (precision == MBH_MIXED)
        return launch_template_mixed(grid, theta_dev, W, (float2*)h_out_dev, (cudaStream_t)stream);
    return fail(MBH_EINVAL, "unknown precision %d", (int)precision);
}

namespace mbh {
mbh_status check_modes(uint32_t modes, mbh_precision precision)
{
    if (modes == 0u || (modes & ~kHmAll)) return fail(MBH_EINVAL, "mode mask 0x%x: bits 0-5, not empty", modes);
    if (precision != MBH_FP64 && precision != MBH_MIXED) return fail(MBH_EINVAL, "unknown precision %d", (int)precision);
    return MBH_OK;
}
}  // namespace mbh

extern "C" mbh_status template_batch_hm(const mbh_grid* grid, const double* theta_dev, int64_t W,
                                        uint32_t modes, mbh_precision precision, void* h_out_dev,
                                        void* stream)
{
    if (mbh_status s = check_modes(modes, precision)) return s;
    if (modes == 1u) return template_batch(grid, theta_dev, W, precision, h_out_dev, stream);
    if (mbh_status s = check_grid(grid)) return s;
    if (W < 0) return fail(MBH_EINVAL, "W < 0");
    if (W == 0) return MBH_OK;
    if (!theta_dev || !h_out_dev) return fail(MBH_EINVAL, "NULL buffer");
    if (mbh_status s = check_device()) return s;
    if (precision == MBH_MIXED)
        return launch_template_mixed(grid, theta_dev, W, (float2*)h_out_dev, (cudaStream_t)stream, modes);
    return launch_template_f64(grid, theta_dev, W, (double2*)h_out_dev, (cudaStream_t)stream, modes);
}

// ------------------------------------------------------------------------------------------
// data
// ------------------------------------------------------------------------------------------
constexpr int kDataThreads = 256;

__global__ void __launch_bounds__(kDataThreads)
    data_kernel(const double2* __restrict__ d, const double* __restrict__ S, int64_t m, double df,
                double sigma, int shift, double2* __restrict__ wd, double* __restrict__ wv,
                float2* __restrict__ wd32, float* __restrict__ wv32, float4* __restrict__ wsp,
                float2* __restrict__ vsp, double* __restrict__ part)
{
    __shared__ double sm[32];
    double acc[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double w = 4.0 * df / S[i];
        const double2 x = d[i];
        wd[i] = make_double2(w * x.x, w * x.y);
        wv[i] = w;
        wd32[i] = make_float2((float)(sigma * w * x.x), (float)(sigma * w * x.y));
        wv32[i] = (float)(sigma * sigma * w);
        // exact float pairs of 2^shift wd and 2^(2 shift) wv for the double-float reduction
        const f2 re = split_f64(w * x.x, -shift), im = split_f64(w * x.y, -shift);
        const f2 vv = split_f64(w, -2 * shift);
        wsp[i] = make_float4(re.hi, im.hi, re.lo, im.lo);
        vsp[i] = make_float2(vv.hi, vv.lo);
        acc[0] += w * (x.x * x.x + x.y * x.y);
    }
    block_sum<1>(acc, sm);
    if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ part, int n, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s;
    }
}

extern "C" mbh_status mbh_data_create(const mbh_grid* grid, const void* d_dev, const double* psd_dev,
                                      void* stream, mbh_data** out)
{
    if (!out) return fail(MBH_EINVAL, "out is NULL");
    *out = nullptr;
    if (mbh_status s = check_grid(grid)) return s;
    if (!d_dev || !psd_dev) return fail(MBH_EINVAL, "NULL buffer");
    if (mbh_status s = check_device()) return s;
    cudaStream_t st = (cudaStream_t)stream;
    dev_status();   // resolve the status word's address here, outside any stream capture
    mbh_data* D = new mbh_data();
    D->grid = *grid;
    cudaGetDevice(&D->device);
    const int64_t m = 3 * grid->n;
    const int nb = grid_blocks(m, kDataThreads);
    double* part = nullptr;
    double* dd_dev = nullptr;
    cudaError_t e = cudaMalloc(&D->wd, sizeof(double2) * m);
    if (e == cudaSuccess) e = cudaMalloc(&D->wv, sizeof(double) * m);
    if (e == cudaSuccess) e = cudaMalloc(&D->wd32, sizeof(float2) * m);
    if (e == cudaSuccess) e = cudaMalloc(&D->wv32, sizeof(float) * m);
    if (e == cudaSuccess) e = cudaMalloc(&D->wsp, sizeof(float4) * m);
    if (e == cudaSuccess) e = cudaMalloc(&D->vsp, sizeof(float2) * m);
    if (e == cudaSuccess) e = cudaMallocAsync(&part, sizeof(double) * (nb + 1), st);
    // scale of the float32 copies: sigma^2 = S_A/(4 df) at the middle of the grid, so that
    // 4 df sigma^2/S and h/sigma are O(1) instead of ~1e40 and ~1e-20
    double s_mid = 0.0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&s_mid, psd_dev + grid->n / 2, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        mbh_data_free(D);
        return cuda_fail(e, "mbh_data_create alloc");
    }
    if (!(s_mid > 0.0) || !std::isfinite(s_mid)) {
        mbh_data_free(D);
        return fail(MBH_EINVAL, "psd must be positive and finite");
    }
    D->sigma = std::sqrt(s_mid / (4.0 * grid->df));
    D->shift = (int)std::lround(std::log2(D->sigma));
    dd_dev = part + nb;
    data_kernel<<<nb, kDataThreads, 0, st>>>((const double2*)d_dev, psd_dev, m, grid->df, D->sigma,
                                             D->shift, D->wd, D->wv, D->wd32, D->wv32, D->wsp,
                                             D->vsp, part);
    if (mbh_status s = make_freq_tables(D, st)) {
        cudaFreeAsync(part, st);
        cudaStreamSynchronize(st);
        mbh_data_free(D);
        return s;
    }
    if (mbh_status s = make_x_direct_tables(D, st)) {
        cudaFreeAsync(part, st);
        cudaStreamSynchronize(st);
        mbh_data_free(D);
        return s;
    }
    sum_partials_kernel<<<1, 32, 0, st>>>(part, nb, dd_dev);
    e = cudaMemcpyAsync(&D->dd, dd_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaFreeAsync(part, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        mbh_data_free(D);
        return cuda_fail(e, "mbh_data_create");
    }
    *out = D;
    return MBH_OK;
}

extern "C" double mbh_data_dd(const mbh_data* data) { return data ? data->dd : NAN; }

extern "C" void mbh_data_free(mbh_data* data)
{
    if (!data) return;
    if (data->wd) cudaFree(data->wd);
    if (data->wv) cudaFree(data->wv);
    if (data->wd32) cudaFree(data->wd32);
    if (data->wv32) cudaFree(data->wv32);
    if (data->wsp) cudaFree(data->wsp);
    if (data->vsp) cudaFree(data->vsp);
    if (data->ftab) cudaFree(data->ftab);
    if (data->ftab2) cudaFree(data->ftab2);
    if (data->ftab3) cudaFree(data->ftab3);
    if (data->wdk) cudaFree(data->wdk);
    if (data->wvk) cudaFree(data->wvk);
    if (data->ftx) cudaFree(data->ftx);
    if (data->ftx2) cudaFree(data->ftx2);
    if (data->wdx) cudaFree(data->wdx);
    if (data->wvx) cudaFree(data->wvx);
    delete data;
}

// ------------------------------------------------------------------------------------------
// direct likelihood
// ------------------------------------------------------------------------------------------
constexpr int kDirThreads = 256;

// Fused generation + reduction, float64.  A grid point's data is loaded once for the T
// walkers; per-thread per-walker sums live in shared memory.
template <int T>
__global__ void __launch_bounds__(kDirThreads)
    direct_fused_f64_kernel(const double* __restrict__ theta, int64_t W, double f0, double df,
                            double t_obs, const double2* __restrict__ wd,
                            const double* __restrict__ wv, int64_t n, int64_t chunk, int nchunks,
                            uint32_t modes, double2* __restrict__ part)
{
    __shared__ Walker ws[T];
    __shared__ double2 acc[T][kDirThreads];
    __shared__ double sm[32 * 2];
    const int64_t w0 = (int64_t)blockIdx.x * T;
    const int ch = blockIdx.y;
    const int nt = (int)std::min<int64_t>(T, W - w0);
    if (threadIdx.x < nt) walker_setup(theta, W, w0 + threadIdx.x, ws[threadIdx.x], modes);
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t][threadIdx.x] = make_double2(0.0, 0.0);
    __syncthreads();
    const int64_t kb = (int64_t)ch * chunk, ke = std::min<int64_t>(n, kb + chunk);
    for (int64_t k = kb + threadIdx.x; k < ke; k += kDirThreads) {
        const double f = f0 + (double)k * df;
        double2 d[3];
        double v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            d[c] = __ldg(wd + (int64_t)c * n + k);
            v[c] = __ldg(wv + (int64_t)c * n + k);
        }
        for (int t = 0; t < nt; ++t) {
            cd h[3];
            if (point_model_f64(ws[t], f, t_obs, h)) {
                double2 s2 = acc[t][threadIdx.x];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    s2.x += d[c].x * h[c].re + d[c].y * h[c].im;
                    s2.y += v[c] * (h[c].re * h[c].re + h[c].im * h[c].im);
                }
                acc[t][threadIdx.x] = s2;
            }
        }
    }
    for (int t = 0; t < nt; ++t) {
        double r[2] = {acc[t][threadIdx.x].x, acc[t][threadIdx.x].y};
        block_sum<2>(r, sm);
        if (threadIdx.x == 0) part[(w0 + t) * nchunks + ch] = make_double2(r[0], r[1]);
    }
}

// lnL = -1/2 (<d|d> + <h|h> - 2 <d|h>), partial sums added in chunk order.
__global__ void direct_finalize_kernel(const double2* __restrict__ part, int nchunks, int64_t W,
                                       double dd, double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= W) return;
    double dh = 0.0, hh = 0.0;
    for (int c = 0; c < nchunks; ++c) {
        const double2 p = part[i * nchunks + c];
        dh += p.x;
        hh += p.y;
    }
    out[i] = -0.5 * (dd + hh - 2.0 * dh);
    out[W + i] = dh;
    out[2 * W + i] = hh;
}

namespace mbh {
// Chunking of the grid for the direct kernels: enough (tile, chunk) blocks for blocks_per_sm
// blocks per SM, chunks of at most max_chunk points.  Every block sets its templates up again,
// so a kernel whose set-up is heavy against a chunk's work (the double-float pass) asks for
// fewer, larger chunks.
void direct_chunks(int64_t n, int64_t tiles, int64_t max_chunk, int64_t& chunk, int& nchunks, int blocks_per_sm)
{
    const int64_t target_blocks = (int64_t)sm_count() * blocks_per_sm;
    int64_t nc = std::max<int64_t>(1, target_blocks / std::max<int64_t>(1, tiles));
    nc = std::max<int64_t>(nc, (n + max_chunk - 1) / max_chunk);
    nc = std::min<int64_t>(nc, (n + kDirThreads - 1) / kDirThreads);
    nc = std::min<int64_t>(nc, 65535);
    chunk = (n + nc - 1) / nc;
    chunk = (chunk + 31) / 32 * 32;
    nchunks = (int)((n + chunk - 1) / chunk);
}

mbh_status direct_finish(double2* part, int nchunks, int64_t W, double dd, double* out,
                         cudaStream_t st)
{
    direct_finalize_kernel<<<(unsigned)((W + 255) / 256), 256, 0, st>>>(part, nchunks, W, dd, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaFreeAsync(part, st);
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "direct finalize");
}
}  // namespace mbh

namespace mbh {
// Final pass of the direct reduction (lnL from the chunk partial sums) into `out`, without
// releasing the partial-sum buffer (for callers that own it).
mbh_status launch_direct_finalize(const double2* part, int nchunks, int64_t W, double dd, double* out,
                                  cudaStream_t st)
{
    direct_finalize_kernel<<<(unsigned)((W + 255) / 256), 256, 0, st>>>(part, nchunks, W, dd, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "direct finalize");
}
}  // namespace mbh

namespace {
mbh_status direct_f64(const mbh_data* data, const double* theta_dev, int64_t W, uint32_t modes,
                      double* out_dev, cudaStream_t st);
}

extern "C" mbh_status direct_loglike_batch_hm(const mbh_data* data, const double* theta_dev, int64_t W,
                                              uint32_t modes, mbh_precision precision, double* out_dev,
                                              void* stream)
{
    // higher modes: MBH_MIXED the double-float pass, MBH_MIXED_F32 the float32-response pass
    if (mbh_status s = check_modes(modes, precision == MBH_MIXED_F32 ? MBH_MIXED : precision)) return s;
    if (modes == 1u) return direct_loglike_batch(data, theta_dev, W, precision, out_dev, stream);
    if (!data) return fail(MBH_EINVAL, "data is NULL");
    if (W < 0) return fail(MBH_EINVAL, "W < 0");
    if (W == 0) return MBH_OK;
    if (!theta_dev || !out_dev) return fail(MBH_EINVAL, "NULL buffer");
    if (precision == MBH_MIXED) return launch_direct_fused_x(data, theta_dev, W, out_dev, (cudaStream_t)stream, modes);
    if (precision == MBH_MIXED_F32)
        return launch_direct_fused_mixed(data, theta_dev, W, out_dev, (cudaStream_t)stream, modes);
    return direct_f64(data, theta_dev, W, modes, out_dev, (cudaStream_t)stream);
}

extern "C" mbh_status direct_loglike_batch(const mbh_data* data, const double* theta_dev, int64_t W,
                                           mbh_precision precision, double* out_dev, void* stream)
{
    if (!data) return fail(MBH_EINVAL, "data is NULL");
    if (W < 0) return fail(MBH_EINVAL, "W < 0");
    if (W == 0) return MBH_OK;
    if (!theta_dev || !out_dev) return fail(MBH_EINVAL, "NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    // MBH_MIXED: the template in double-float at every point (extended-precision pass);
    // MBH_MIXED_F32: double-float phase, float32 response and products
    if (precision == MBH_MIXED) return launch_direct_fused_x(data, theta_dev, W, out_dev, st);
    if (precision == MBH_MIXED_F32) return launch_direct_fused_mixed(data, theta_dev, W, out_dev, st);
    if (precision != MBH_FP64) return fail(MBH_EINVAL, "unknown precision %d", (int)precision);
    return direct_f64(data, theta_dev, W, 1u, out_dev, st);
}

namespace {
mbh_status direct_f64(const mbh_data* data, const double* theta_dev, int64_t W, uint32_t modes,
                      double* out_dev, cudaStream_t st)
{
    constexpr int T = 4;
    const int64_t tiles = (W + T - 1) / T;
    if (tiles > 0x7fffffff) return fail(MBH_EINVAL, "W too large");
    int64_t chunk;
    int nchunks;
    direct_chunks(data->grid.n, tiles, 1 << 14, chunk, nchunks);
    double2* part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, sizeof(double2) * W * nchunks, st);
    if (e != cudaSuccess) return cuda_fail(e, "direct_loglike_batch alloc");
    dim3 grid((unsigned)tiles, (unsigned)nchunks);
    direct_fused_f64_kernel<T><<<grid, kDirThreads, 0, st>>>(theta_dev, W, data->grid.f0, data->grid.df,
                                                            data->grid.t_obs, data->wd, data->wv,
                                                            data->grid.n, chunk, nchunks, modes, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "direct_loglike_batch");
    return direct_finish(part, nchunks, W, data->dd, out_dev, st);
}
}  // namespace

// ------------------------------------------------------------------------------------------
// heterodyne: reference preparation
// ------------------------------------------------------------------------------------------
constexpr int kPrepThreads = 256;
constexpr int64_t kPrepItem = 2048;   // grid points per (bin, sub-range) item

__global__ void band_kernel(const double* __restrict__ theta0, double f0, double df, int64_t n,
                            double t_obs, uint32_t modes, unsigned long long* __restrict__ kminmax)
{
    __shared__ Walker w;
    if (threadIdx.x == 0) walker_setup(theta0, 1, 0, w, modes);
    __syncthreads();
    unsigned long long lo = ~0ull, hi = 0ull;
    bool any = false;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (support_model_f64(w, f0 + (double)k * df, t_obs)) {
            lo = std::min<unsigned long long>(lo, (unsigned long long)k);
            hi = std::max<unsigned long long>(hi, (unsigned long long)k);
            any = true;
        }
    }
    if (any) {
        atomicMin(&kminmax[0], lo);
        atomicMax(&kminmax[1], hi);
    }
}

// One block per item = (bin, [k0, k1)): float64 reference template and the 18 per-bin sums
// (per channel: Re/Im of sum wd conj(h0), Re/Im of sum wd conj(h0)(f - f_b), sum wv |h0|^2,
// sum wv |h0|^2 (f - f_b)), with wd = 4 df d/S, wv = 4 df/S; the factor 1/4 is applied at
// the end so that A0 = sum d conj(h0)/S df etc.
__global__ void __launch_bounds__(kPrepThreads)
    prep_items_kernel(const double* __restrict__ theta0, double f0, double df, int64_t n,
                      double t_obs, const double2* __restrict__ wd, const double* __restrict__ wv,
                      const PrepItem* __restrict__ items, const double* __restrict__ fb,
                      uint32_t modes, double* __restrict__ part)
{
    __shared__ Walker w;
    __shared__ double sm[32 * 18];
    if (threadIdx.x == 0) walker_setup(theta0, 1, 0, w, modes);
    __syncthreads();
    const PrepItem it = items[blockIdx.x];
    const double fbin = fb[it.bin];
    double acc[18];
#pragma unroll
    for (int j = 0; j < 18; ++j) acc[j] = 0.0;
    for (int64_t k = it.k0 + threadIdx.x; k < it.k1; k += kPrepThreads) {
        const double f = f0 + (double)k * df;
        cd h[3];
        if (!point_model_f64(w, f, t_obs, h)) continue;
        const double x = f - fbin;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 d = wd[(int64_t)c * n + k];
            const double v = wv[(int64_t)c * n + k];
            const double re = d.x * h[c].re + d.y * h[c].im;   // Re(d conj h)
            const double im = d.y * h[c].re - d.x * h[c].im;   // Im(d conj h)
            const double hh = v * (h[c].re * h[c].re + h[c].im * h[c].im);
            acc[6 * c + 0] += re;
            acc[6 * c + 1] += im;
            acc[6 * c + 2] += re * x;
            acc[6 * c + 3] += im * x;
            acc[6 * c + 4] += hh;
            acc[6 * c + 5] += hh * x;
        }
    }
    block_sum<18>(acc, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int j = 0; j < 18; ++j) part[(int64_t)blockIdx.x * 18 + j] = acc[j];
}

// summary[b][c][m] = 1/4 sum over the items of bin b, in order.
__global__ void prep_finalize_kernel(const double* __restrict__ part,
                                     const int32_t* __restrict__ item_begin, int E,
                                     double* __restrict__ summary)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E * 18) return;
    const int b = i / 18, j = i % 18;
    double s = 0.0;
    for (int it = item_begin[b]; it < item_begin[b + 1]; ++it) s += part[(int64_t)it * 18 + j];
    summary[(int64_t)b * 18 + j] = 0.25 * s;
}

// Reference template at the bin edges: h0 and 1/h0 (0 where h0 = 0), plus the factored form
// used by the mixed kernel (float64 large phase and the float32 transfer).
__global__ void edge_ref_kernel(const double* __restrict__ theta0, double t_obs,
                                const double* __restrict__ fe, int n_edges, uint32_t modes,
                                double2* __restrict__ h0e, double2* __restrict__ h0inv)
{
    __shared__ Walker w;
    if (threadIdx.x == 0) walker_setup(theta0, 1, 0, w, modes);
    __syncthreads();
    for (int e = threadIdx.x; e < n_edges; e += blockDim.x) {
        cd h[3];
        point_model_f64(w, fe[e], t_obs, h);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h0e[e * 3 + c] = make_double2(h[c].re, h[c].im);
            const double m2 = h[c].re * h[c].re + h[c].im * h[c].im;
            h0inv[e * 3 + c] = m2 > 0.0 ? make_double2(h[c].re / m2, -h[c].im / m2)
                                        : make_double2(0.0, 0.0);
        }
    }
}

namespace mbh {
// Log-spaced edges over [kmin, kmax] (Sec. III B): targets f_lo (f_hi/f_lo)^{b/B} rounded to
// the nearest grid index, endpoints exact, duplicates dropped.
std::vector<int64_t> make_edges(int64_t kmin, int64_t kmax, int nbins, double f0, double df)
{
    std::vector<int64_t> e;
    const double flo = f0 + (double)kmin * df, fhi = f0 + (double)kmax * df;
    for (int b = 0; b <= nbins; ++b) {
        int64_t k;
        if (b == 0)
            k = kmin;
        else if (b == nbins)
            k = kmax;
        else {
            const double ft = flo * std::pow(fhi / flo, (double)b / nbins);
            k = std::llround((ft - f0) / df);
            k = std::min(std::max(k, kmin), kmax);
        }
        if (e.empty() || k > e.back()) e.push_back(k);
    }
    return e;
}
}  // namespace mbh

extern "C" mbh_status het_prepare_reference(const mbh_data* data, const double* theta0_host,
                                            int32_t n_bins, void* stream, mbh_ref** out)
{
    return het_prepare_reference_hm(data, theta0_host, n_bins, 1u, stream, out);
}

extern "C" mbh_status het_prepare_reference_hm(const mbh_data* data, const double* theta0_host,
                                               int32_t n_bins, uint32_t modes, void* stream,
                                               mbh_ref** out)
{
    if (!out) return fail(MBH_EINVAL, "out is NULL");
    if (modes == 0u || (modes & ~kHmAll)) return fail(MBH_EINVAL, "mode mask 0x%x: bits 0-5, not empty", modes);
    *out = nullptr;
    if (!data || !theta0_host) return fail(MBH_EINVAL, "NULL argument");
    if (n_bins < 1 || n_bins > kMaxBins) return fail(MBH_EINVAL, "n_bins %d outside [1, %d]", n_bins, kMaxBins);
    for (int j = 0; j < kNParams; ++j)
        if (!std::isfinite(theta0_host[j])) return fail(MBH_EINVAL, "theta0[%d] not finite", j);
    if (!(theta0_host[kMT] > 0.0) || !(theta0_host[kQ] > 0.0) || !(theta0_host[kDL] > 0.0))
        return fail(MBH_EINVAL, "theta0 needs M_T, q, D_L > 0");
    cudaStream_t st = (cudaStream_t)stream;
    const mbh_grid& g = data->grid;
    dev_status();   // resolve the status word's address here, outside any stream capture
    mbh_ref* R = new mbh_ref();
    R->modes = modes;
    R->grid = g;
    R->dd = data->dd;
    std::memcpy(R->theta0, theta0_host, sizeof(R->theta0));
    cudaGetDevice(&R->device);
    auto bail = [&](cudaError_t e, const char* where) {
        mbh_ref_free(R);
        return cuda_fail(e, where);
    };
    cudaError_t e = cudaMalloc(&R->theta0_dev, sizeof(double) * kNParams);
    if (e != cudaSuccess) return bail(e, "prepare alloc");
    e = cudaMemcpyAsync(R->theta0_dev, theta0_host, sizeof(double) * kNParams, cudaMemcpyHostToDevice, st);
    unsigned long long* kmm = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&kmm, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(kmm, 0xff, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(kmm + 1, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return bail(e, "prepare setup");
    band_kernel<<<grid_blocks(g.n, 256), 256, 0, st>>>(R->theta0_dev, g.f0, g.df, g.n, g.t_obs, modes, kmm);
    unsigned long long h_kmm[2];
    e = cudaMemcpyAsync(h_kmm, kmm, sizeof h_kmm, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaFreeAsync(kmm, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(e, "prepare band");
    if (h_kmm[0] == ~0ull || h_kmm[1] <= h_kmm[0]) {
        mbh_ref_free(R);
        return fail(MBH_EINVAL, "reference band has fewer than two grid points");
    }
    R->band[0] = (int64_t)h_kmm[0];
    R->band[1] = (int64_t)h_kmm[1];
    R->edges_host = make_edges(R->band[0], R->band[1], n_bins, g.f0, g.df);
    const int E = (int)R->edges_host.size() - 1;
    R->E = E;

    // host-side tables: edge frequencies, bin centres and widths, items
    std::vector<double> fe(E + 1), fb(E), invw(E);
    for (int i = 0; i <= E; ++i) fe[i] = g.f0 + (double)R->edges_host[i] * g.df;
    for (int b = 0; b < E; ++b) {
        fb[b] = 0.5 * (fe[b] + fe[b + 1]);
        invw[b] = 1.0 / (fe[b + 1] - fe[b]);
    }
    std::vector<PrepItem> items;
    std::vector<int32_t> item_begin(E + 1);
    for (int b = 0; b < E; ++b) {
        item_begin[b] = (int32_t)items.size();
        const int64_t k0 = R->edges_host[b];
        const int64_t k1 = (b == E - 1) ? R->edges_host[b + 1] + 1 : R->edges_host[b + 1];
        for (int64_t k = k0; k < k1; k += kPrepItem) items.push_back({b, k, std::min(k1, k + kPrepItem)});
    }
    item_begin[E] = (int32_t)items.size();
    const int nitems = (int)items.size();

    e = alloc_ref_tables(R);
    if (e != cudaSuccess) return bail(e, "prepare alloc tables");
    PrepItem* d_items = nullptr;
    int32_t* d_ib = nullptr;
    double *d_fb = nullptr, *d_part = nullptr;
    e = cudaMallocAsync(&d_items, sizeof(PrepItem) * nitems, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_ib, sizeof(int32_t) * (E + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_fb, sizeof(double) * E, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_part, sizeof(double) * 18 * (size_t)nitems, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_items, items.data(), sizeof(PrepItem) * nitems, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ib, item_begin.data(), sizeof(int32_t) * (E + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_fb, fb.data(), sizeof(double) * E, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R->edges, R->edges_host.data(), sizeof(int64_t) * (E + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R->fe, fe.data(), sizeof(double) * (E + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R->invw, invw.data(), sizeof(double) * E, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return bail(e, "prepare upload");

    prep_items_kernel<<<nitems, kPrepThreads, 0, st>>>(R->theta0_dev, g.f0, g.df, g.n, g.t_obs, data->wd,
                                                        data->wv, d_items, d_fb, modes, d_part);
    prep_finalize_kernel<<<(E * 18 + 255) / 256, 256, 0, st>>>(d_part, d_ib, E, R->summary);
    edge_ref_kernel<<<1, 256, 0, st>>>(R->theta0_dev, g.t_obs, R->fe, E + 1, modes, R->h0e, R->h0inv);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = prepare_mixed_tables(R, st);
    if (e == cudaSuccess) e = modes == 1u ? prepare_x_tables(R, st) : prepare_x_tables_hm(R, st);
    if (e == cudaSuccess) e = cudaFreeAsync(d_items, st);
    if (e == cudaSuccess) e = cudaFreeAsync(d_ib, st);
    if (e == cudaSuccess) e = cudaFreeAsync(d_fb, st);
    if (e == cudaSuccess) e = cudaFreeAsync(d_part, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(e, "prepare kernels");
    *out = R;
    return MBH_OK;
}

extern "C" int32_t mbh_ref_bins(const mbh_ref* ref) { return ref ? ref->E : -1; }
extern "C" uint32_t mbh_ref_modes(const mbh_ref* ref) { return ref ? ref->modes : 0u; }
extern "C" int32_t mbh_ref_f32_edges(const mbh_ref* ref) { return ref ? ref->mix.xn32 : -1; }

extern "C" mbh_status mbh_ref_read(const mbh_ref* ref, int64_t* edges_host, double* summary_host,
                                   double* h0_edges_host, double* dd_host)
{
    if (!ref) return fail(MBH_EINVAL, "ref is NULL");
    if (edges_host) std::memcpy(edges_host, ref->edges_host.data(), sizeof(int64_t) * (ref->E + 1));
    cudaError_t e = cudaSuccess;
    if (summary_host)
        e = cudaMemcpy(summary_host, ref->summary, sizeof(double) * 18 * ref->E, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h0_edges_host)
        e = cudaMemcpy(h0_edges_host, ref->h0e, sizeof(double2) * 3 * (ref->E + 1), cudaMemcpyDeviceToHost);
    if (dd_host) *dd_host = ref->dd;
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "mbh_ref_read");
}

extern "C" void mbh_ref_free(mbh_ref* ref)
{
    if (!ref) return;
    free_ref_tables(ref);
    if (ref->theta0_dev) cudaFree(ref->theta0_dev);
    delete ref;
}

// ------------------------------------------------------------------------------------------
// heterodyne: likelihood, float64
// ------------------------------------------------------------------------------------------
// G threads per walker, BLOCK/G walkers per block; a block's walkers share one source.  Edges
// are dealt round-robin: in round r lane j evaluates edge e = r G + j; bin e-1 pairs it with
// edge e-1, taken from lane j-1 by a shuffle (lane 0 keeps the previous round's last edge).
template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    het_f64_kernel(const __grid_constant__ HetLaunch L)
{
    constexpr int WPB = BLOCK / G;
    __shared__ Walker ws[WPB];
    const int lw = threadIdx.x / G, lane = threadIdx.x % G;
    for (int tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
        int s = 0;
        while (s + 1 < L.n_src && L.src[s + 1].tile_begin <= tile) ++s;
        const SrcDesc& S = L.src[s];
        const int64_t wi = S.w_begin + (int64_t)(tile - S.tile_begin) * WPB + lw;
        const bool active = wi < S.w_end;
        __syncthreads();
        if (lane == 0 && active) walker_setup(L.theta, L.W, wi, ws[lw], S.modes);
        __syncthreads();
        const int E = S.E;
        double dh = 0.0, hh = 0.0;
        cd carry[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        const int rounds = (E + 1 + G - 1) / G;
        for (int r = 0; r < rounds; ++r) {
            const int e = r * G + lane;
            cd rr[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
            const bool ok = active && e <= E && MBH_IN_RANGE(L.status, e, (long long)S.E_check + 1, kKernHetF64, s);
            if (ok) {
                cd h[3];
                if (point_model_f64(ws[lw], S.fe[e], S.t_obs, h)) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const double2 iv = S.h0inv[e * 3 + c];
                        rr[c] = cmul(h[c], {iv.x, iv.y});
                    }
                }
            }
            cd rp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rp[c].re = __shfl_up_sync(0xffffffffu, rr[c].re, 1, G);
                rp[c].im = __shfl_up_sync(0xffffffffu, rr[c].im, 1, G);
                if (lane == 0) rp[c] = carry[c];
                carry[c].re = __shfl_sync(0xffffffffu, rr[c].re, G - 1, G);
                carry[c].im = __shfl_sync(0xffffffffu, rr[c].im, G - 1, G);
            }
            if (ok && e >= 1) {
                const int b = e - 1;
                const double iw = S.invw[b];
                const double* sm = S.summary + (int64_t)b * 18;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const cd r0 = {0.5 * (rp[c].re + rr[c].re), 0.5 * (rp[c].im + rr[c].im)};
                    const cd r1 = {(rr[c].re - rp[c].re) * iw, (rr[c].im - rp[c].im) * iw};
                    const double* q = sm + 6 * c;
                    dh += q[0] * r0.re + q[1] * r0.im + q[2] * r1.re + q[3] * r1.im;
                    hh += q[4] * (r0.re * r0.re + r0.im * r0.im) +
                          2.0 * q[5] * (r0.re * r1.re + r0.im * r1.im);
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            dh += __shfl_down_sync(0xffffffffu, dh, o, G);
            hh += __shfl_down_sync(0xffffffffu, hh, o, G);
        }
        if (active && lane == 0) {
            dh *= 4.0;
            hh *= 4.0;
            L.out[wi] = -0.5 * (S.dd + hh - 2.0 * dh);
            L.out[L.W + wi] = dh;
            L.out[2 * L.W + wi] = hh;
        }
    }
}

namespace {
template <int G, int BLOCK>
cudaError_t launch_het_f64(const HetLaunch& L, int grid, cudaStream_t st)
{
    het_f64_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}
}  // namespace

namespace mbh {
HetKernel het_kernel_f64(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return {&launch_het_f64<g, b>, (const void*)&het_f64_kernel<g, b>};
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

// Direct likelihood of stored templates (Katz, arXiv:2111.01064, Sec. II, Eqs. 2-3): the
// HBM-bound streaming reduction <d|h> = sum Re(conj(4 df d/S) h), <h|h> = sum 4 df/S |h|^2
// over 3 channels x n frequencies per template.
//
//   direct_stored_df_kernel   complex128 templates, float64-class accuracy from double-float
//                             arithmetic on the float32/integer pipes (mbh_df.cuh): B300's
//                             float64 pipe (2 FMA/SM/clock) would cap this reduction at
//                             ~1.8 TB/s, the double-float form leaves it HBM-bound.
//   direct_stored_f32_kernel  complex64 templates, float32 products on O(1)-scaled operands,
//                             float64 sums.
// Block = (walker tile of T templates, frequency chunk); the data of a chunk is read once per
// block and reused by its T templates, and walker tiles vary fastest in launch order so the
// tiles sharing a chunk run together and find the data in L2.  Per-block partial sums go to a
// scratch array, added in chunk order by direct_finalize_kernel (deterministic).
#include <cuda_runtime.h>

#include <algorithm>

#include "mbh_df.cuh"
#include "mbh_internal.cuh"

using namespace mbh;

constexpr int kStreamThreads = 256;

// Block-wide double-float sum of N values (shuffles of hi/lo with the two-sum); the result,
// converted to float64, is valid in thread 0.  No float64 arithmetic per thread.
template <int N>
__device__ void block_sum_df(f2 (&v)[N], double (&out)[N])
{
    __shared__ float2 sm[N][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            df_acc(v[j], {__shfl_down_sync(0xffffffffu, v[j].hi, o), __shfl_down_sync(0xffffffffu, v[j].lo, o)});
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < N; ++j) sm[j][warp] = make_float2(v[j].hi, v[j].lo);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            f2 x = lane < nw ? f2{sm[j][lane].x, sm[j][lane].y} : f2{0.0f, 0.0f};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                df_acc(x, {__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)});
            out[j] = df_to_double(x);
        }
    }
}

// U grid points per thread per step, loads for all of them (data pair + T templates) issued
// before any arithmetic, so that enough bytes are in flight to cover HBM latency.
template <int T, int U>
__global__ void __launch_bounds__(kStreamThreads)
    direct_stored_df_kernel(const float4* __restrict__ wsp, const float2* __restrict__ vsp,
                            const double2* __restrict__ h, int64_t n, int64_t W, int64_t chunk,
                            int nchunks, int shift, double2* __restrict__ part)
{
    const int64_t w0 = (int64_t)blockIdx.x * T;
    const int ch = blockIdx.y;
    const int64_t kb = (int64_t)ch * chunk, ke = std::min<int64_t>(n, kb + chunk);
    const int nt = (int)std::min<int64_t>(T, W - w0);
    f2 adh[T], ahh[T];
#pragma unroll
    for (int t = 0; t < T; ++t) adh[t] = ahh[t] = {0.0f, 0.0f};
    for (int c = 0; c < 3; ++c) {
        const float4* wc = wsp + (int64_t)c * n;
        const float2* vc = vsp + (int64_t)c * n;
        const double2* hc = h + (w0 * 3 + c) * n;
        for (int64_t k0 = kb + threadIdx.x; k0 < ke; k0 += (int64_t)U * kStreamThreads) {
            float4 d[U];
            float2 v2[U];
            double2 x[U][T];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = k0 + (int64_t)u * kStreamThreads;
                const bool ok = k < ke;
                d[u] = ok ? __ldg(wc + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                v2[u] = ok ? __ldg(vc + k) : make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < T; ++t)
                    x[u][t] = (ok && t < nt) ? __ldcs(hc + (int64_t)t * 3 * n + k) : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const f2 dre = {d[u].x, d[u].z}, dim = {d[u].y, d[u].w}, v = {v2[u].x, v2[u].y};
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const f2 xr = split_f64(x[u][t].x, shift), xi = split_f64(x[u][t].y, shift);
                    df_acc(adh[t], df_mul(dre, xr));
                    df_acc(adh[t], df_mul(dim, xi));
                    df_acc(ahh[t], df_mul(v, df_add(df_sqr(xr), df_sqr(xi))));
                }
            }
        }
    }
    f2 vals[2 * T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        vals[2 * t] = adh[t];
        vals[2 * t + 1] = ahh[t];
    }
    double acc[2 * T];
    block_sum_df<2 * T>(vals, acc);
    if (threadIdx.x == 0)
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (t < nt) part[(w0 + t) * nchunks + ch] = make_double2(acc[2 * t], acc[2 * t + 1]);
}

// complex64 templates: loads of U grid points issued before the arithmetic; float32 products
// on O(1)-scaled operands, float32 sums per channel pass, float64 across passes.
template <int T, int U>
__global__ void __launch_bounds__(kStreamThreads)
    direct_stored_f32_kernel(const float2* __restrict__ wd, const float* __restrict__ wv,
                             const float2* __restrict__ h, int64_t n, int64_t W, int64_t chunk,
                             int nchunks, float inv_sigma, double2* __restrict__ part)
{
    __shared__ double sm[32 * 2 * T];
    const int64_t w0 = (int64_t)blockIdx.x * T;
    const int ch = blockIdx.y;
    const int64_t kb = (int64_t)ch * chunk, ke = std::min<int64_t>(n, kb + chunk);
    const int nt = (int)std::min<int64_t>(T, W - w0);
    double acc[2 * T];
#pragma unroll
    for (int t = 0; t < 2 * T; ++t) acc[t] = 0.0;
    for (int c = 0; c < 3; ++c) {
        const float2* wc = wd + (int64_t)c * n;
        const float* vc = wv + (int64_t)c * n;
        const float2* hc = h + (w0 * 3 + c) * n;
        float pd[T], ph[T];
#pragma unroll
        for (int t = 0; t < T; ++t) pd[t] = ph[t] = 0.0f;
        for (int64_t k0 = kb + threadIdx.x; k0 < ke; k0 += (int64_t)U * kStreamThreads) {
            float2 d[U];
            float v[U];
            float2 x[U][T];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = k0 + (int64_t)u * kStreamThreads;
                const bool ok = k < ke;
                d[u] = ok ? __ldg(wc + k) : make_float2(0.f, 0.f);
                v[u] = ok ? __ldg(vc + k) : 0.0f;
#pragma unroll
                for (int t = 0; t < T; ++t)
                    x[u][t] = (ok && t < nt) ? __ldcs(hc + (int64_t)t * 3 * n + k) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    const float xr = x[u][t].x * inv_sigma, xi = x[u][t].y * inv_sigma;
                    pd[t] = fmaf(d[u].x, xr, fmaf(d[u].y, xi, pd[t]));
                    ph[t] = fmaf(v[u], fmaf(xr, xr, xi * xi), ph[t]);
                }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            acc[2 * t] += (double)pd[t];
            acc[2 * t + 1] += (double)ph[t];
        }
    }
    block_sum<2 * T>(acc, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (t < nt) part[(w0 + t) * nchunks + ch] = make_double2(acc[2 * t], acc[2 * t + 1]);
}

namespace mbh {
// Launch the stored-template reduction into caller-provided partial sums part[W][nchunks].
mbh_status launch_stored(const mbh_data* data, const void* h, int64_t W, mbh_precision p,
                         double2* part, int64_t chunk, int nchunks, cudaStream_t st)
{
    constexpr int T = 4;
    const int64_t tiles = (W + T - 1) / T;
    dim3 grid((unsigned)tiles, (unsigned)nchunks);
    if (p == MBH_FP64)
        direct_stored_df_kernel<T, 4><<<grid, kStreamThreads, 0, st>>>(
            data->wsp, data->vsp, (const double2*)h, data->grid.n, W, chunk, nchunks, data->shift, part);
    else
        direct_stored_f32_kernel<T, 4><<<grid, kStreamThreads, 0, st>>>(
            data->wd32, data->wv32, (const float2*)h, data->grid.n, W, chunk, nchunks,
            (float)(1.0 / data->sigma), part);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "direct_stored kernel");
}

mbh_status stored_plan(const mbh_data* data, int64_t W, int64_t& chunk, int& nchunks)
{
    constexpr int T = 4;
    const int64_t tiles = (W + T - 1) / T;
    if (tiles > 0x7fffffff) return fail(MBH_EINVAL, "W too large");
    // about two waves of (tile, chunk) blocks, each thread reducing >= 16 points per channel
    const int64_t min_chunk = 16 * kStreamThreads;
    int64_t nc = std::max<int64_t>(1, ((int64_t)sm_count() * 16) / std::max<int64_t>(1, tiles));
    nc = std::min<int64_t>(nc, std::max<int64_t>(1, data->grid.n / min_chunk));
    nc = std::max<int64_t>(nc, (data->grid.n + (1 << 18) - 1) / (1 << 18));
    nc = std::min<int64_t>(nc, 65535);
    chunk = (data->grid.n + nc - 1) / nc;
    chunk = (chunk + 31) / 32 * 32;
    nchunks = (int)((data->grid.n + chunk - 1) / chunk);
    return MBH_OK;
}
}  // namespace mbh

extern "C" mbh_status direct_loglike_stored(const mbh_data* data, const void* h_dev, int64_t W,
                                            mbh_precision precision, double* out_dev, void* stream)
{
    if (!data) return fail(MBH_EINVAL, "data is NULL");
    if (W < 0) return fail(MBH_EINVAL, "W < 0");
    if (W == 0) return MBH_OK;
    if (!h_dev || !out_dev) return fail(MBH_EINVAL, "NULL buffer");
    if (precision != MBH_FP64 && precision != MBH_MIXED)
        return fail(MBH_EINVAL, "unknown precision %d", (int)precision);
    cudaStream_t st = (cudaStream_t)stream;
    int64_t chunk;
    int nchunks;
    if (mbh_status s = stored_plan(data, W, chunk, nchunks)) return s;
    double2* part = nullptr;
    cudaError_t e = cudaMallocAsync(&part, sizeof(double2) * W * nchunks, st);
    if (e != cudaSuccess) return cuda_fail(e, "direct_loglike_stored alloc");
    if (mbh_status s = launch_stored(data, h_dev, W, precision, part, chunk, nchunks, st)) {
        cudaFreeAsync(part, st);
        return s;
    }
    return direct_finish(part, nchunks, W, data->dd, out_dev, st);
}

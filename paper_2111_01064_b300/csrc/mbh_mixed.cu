// Mixed-precision path of libmbhlike (Katz, arXiv:2111.01064, Sec. II): the large phases
// Phi(f) = Psi(f) + 2 pi f k.c(t(f)) (up to ~1e7 rad) and t(f) stay float64; amplitudes, the
// response, ratios and products are float32; sums are float64.
//
// B300 runs float64 FMA at ~1/61 of the float32 rate and float64 sin/log far slower still,
// so the float64 part is cut to multiply-adds:
//  - v = (pi M f)^{1/3} and ln v come from per-frequency tables (f^{1/3}, f^{-1/3}, ln f / 3)
//    times per-walker constants, so no float64 cbrt/log per point;
//  - the orbital angle alpha(t) = alpha(t_ref) + dalpha with dalpha = 2 pi (t - t_ref)/yr:
//    sin/cos alpha(t_ref) are float64 per walker and the correction
//    (cos dalpha - 1, sin dalpha) is float32 from the half angle, accurate relative to its
//    own (small) size, then added in float64;
//  - the phase is reduced modulo 2 pi in float64 and only then rounded to float32.
// The heterodyne works in delta = r - 1 = (rho - 1) e^{-i dPhi} + (e^{-i dPhi} - 1), with
// rho = H/H0 the float32 ratio of the transfer parts and dPhi = Phi - Phi0 in float64, and
// contracts the "1" part once in float64 (sum Re A0, sum B0).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "mbh_internal.cuh"
#include "mbh_model.cuh"

using namespace mbh;

namespace mbh {

std::mutex& launch_mutex()
{
    static std::mutex m;
    return m;
}

struct cf { float re, im; };
__device__ __forceinline__ cf fmul(cf a, cf b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf fadd(cf a, cf b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf fsub(cf a, cf b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cf fscale(cf a, float s) { return {a.re * s, a.im * s}; }

// float32 copies of the response constants of a walker
struct WalkerF {
    float k[3], Pp[6], Pc[6], Kp[2], Kc[2];
    float sa_ref, ca_ref, amp, inv_fc2;
};

__device__ inline void walker_f32(const Walker& w, WalkerF& m)
{
#pragma unroll
    for (int j = 0; j < 3; ++j) m.k[j] = (float)w.k[j];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        m.Pp[j] = (float)w.Pp[j];
        m.Pc[j] = (float)w.Pc[j];
    }
    m.Kp[0] = (float)w.Kp[0];
    m.Kp[1] = (float)w.Kp[1];
    m.Kc[0] = (float)w.Kc[0];
    m.Kc[1] = (float)w.Kc[1];
    m.sa_ref = (float)w.sa_ref;
    m.ca_ref = (float)w.ca_ref;
    m.amp = (float)w.amp;
    m.inv_fc2 = (float)w.inv_fc2;
}

__device__ __forceinline__ float nPnf(const float* P, const float* n)
{
    return P[0] * n[0] * n[0] + P[3] * n[1] * n[1] + P[5] * n[2] * n[2] +
           2.0f * (P[1] * n[0] * n[1] + P[2] * n[0] * n[2] + P[4] * n[1] * n[2]);
}

__device__ __forceinline__ float sincf(float x) { return x == 0.0f ? 1.0f : sinf(x) / x; }

// sinc(x (1 + k)) - sinc(x (1 - k)) without cancellation: for arguments below 1 as
// (a^2 - b^2) sum_{j>=1} (-1)^j P_j / (2j+1)!, P_1 = 1, P_{j+1} = a^2 P_j + b^{2j}
// (a^{2j} - b^{2j} = (a^2 - b^2) P_j), with a^2 - b^2 = 4 x^2 k; directly above.
__device__ __forceinline__ float sinc_diff(float x, float k)
{
    const float a = x * (1.0f + k), b = x * (1.0f - k);
    if (fmaxf(fabsf(a), fabsf(b)) >= 1.0f) return sincf(a) - sincf(b);
    const float a2 = a * a, b2 = b * b;
    // 1/(2j+1)! for j = 1..7
    const float inv_fact[7] = {1.0f / 6.0f, 1.0f / 120.0f, 1.0f / 5040.0f, 1.0f / 362880.0f,
                               1.0f / 39916800.0f, 1.0f / 6227020800.0f, 1.0f / 1307674368000.0f};
    float P = 1.0f, bp = 1.0f, sum = 0.0f, sign = -1.0f;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        sum += sign * P * inv_fact[j];
        sign = -sign;
        bp *= b2;
        P = a2 * P + bp;
    }
    return 4.0f * x * x * k * sum;
}

// Transfer T_c(f) in float32: the construction of transfer_f64, rearranged so that no
// step cancels to leading order at small f L (which float32 cannot afford):
//   1 - D = 2i sin x e^{-ix}, 1 - D^2 = 2i sin 2x e^{-2ix} (no 1 - cos), and
//   X + Y + Z = (1 - D^2)(1 - D) sum_arms g_a [sinc(x(1 + k.n)) - sinc(x(1 - k.n))],
// so T = (X + Y + Z)/sqrt3 is formed from sinc differences computed without cancellation.
__device__ inline void transfer_f32(const WalkerF& w, float f, float sa, float ca, cf T[3])
{
    constexpr float armS = (float)kArmSec;
    constexpr float rho = (float)(kArmSec / kSqrt3);
    constexpr float h3 = (float)(0.5 * kSqrt3);
    const float sp[3] = {sa, -0.5f * sa - h3 * ca, -0.5f * sa + h3 * ca};
    const float cp[3] = {ca, -0.5f * ca + h3 * sa, -0.5f * ca - h3 * sa};
    float o[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o[i][0] = rho * (-sp[i] * sa - 0.5f * cp[i] * ca);
        o[i][1] = rho * (sp[i] * ca - 0.5f * cp[i] * sa);
        o[i][2] = -rho * h3 * cp[i];
    }
    const float x = (float)kPi * armS * f;
    cf yf[3], yb[3], tsum = {0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = a, j = (a + 1) % 3;
        float n[3], kn = 0.0f, ko = 0.0f;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            n[m] = (o[j][m] - o[i][m]) * (1.0f / armS);
            kn += w.k[m] * n[m];
            ko += w.k[m] * (o[i][m] + o[j][m]);
        }
        const float np = nPnf(w.Pp, n), nc = nPnf(w.Pc, n);
        const cf F = {np * w.Kp[0] + nc * w.Kc[0], np * w.Kp[1] + nc * w.Kc[1]};
        float sph, cph;
        sincosf((float)kPi * f * (armS + ko), &sph, &cph);
        const cf g = fmul({-x * sph, -x * cph}, F);
        yf[a] = fscale(g, sincf(x * (1.0f - kn)));
        yb[a] = fscale(g, sincf(x * (1.0f + kn)));
        tsum = fadd(tsum, fscale(g, sinc_diff(x, kn)));   // y_{j->i} - y_{i->j}
    }
    const cf y12 = yf[0], y21 = yb[0], y23 = yf[1], y32 = yb[1], y31 = yf[2], y13 = yb[2];
    float s1, c1;
    sincosf(x, &s1, &c1);
    const float s2 = 2.0f * s1 * c1, c2 = 1.0f - 2.0f * s1 * s1;   // sin 2x, cos 2x
    const cf D = {c2, -s2};
    const cf W1 = {2.0f * s1 * s1, 2.0f * s1 * c1};                 // 1 - D
    const cf W2 = {2.0f * s2 * s2, 2.0f * s2 * c2};                 // 1 - D^2
    const cf X = fmul(W2, fsub(fadd(y21, fmul(D, y12)), fadd(y31, fmul(D, y13))));
    const cf Y = fmul(W2, fsub(fadd(y32, fmul(D, y23)), fadd(y12, fmul(D, y21))));
    const cf Z = fmul(W2, fsub(fadd(y13, fmul(D, y31)), fadd(y23, fmul(D, y32))));
    T[0] = fscale(fsub(Z, X), (float)(1.0 / kSqrt2));
    T[1] = fscale(fadd(fsub(X, fscale(Y, 2.0f)), Z), (float)(1.0 / kSqrt6));
    T[2] = fscale(fmul(fmul(W2, W1), tsum), (float)(1.0 / kSqrt3));
}

// Float64 large phase Phi(f) and float32 amplitude, orbit angle, from the frequency tables.
// Returns false outside the support (f > f_cut or t(f) outside [0, t_obs]).
__device__ __forceinline__ bool phase_mixed(const Walker& w, const WalkerF& wf, double f, double f3,
                                            double fm3, double lnf3, double t_obs, double& Phi,
                                            float& sa, float& ca, float& amp)
{
    const double v = w.cbrt_piM * f3;
    const double iv = w.icbrt_piM * fm3;
    const double lnv = w.ln_cbrt_piM + lnf3;
    double P = w.c[7], Q = w.d[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) {
        P = fma(P, v, w.c[k]);
        Q = fma(Q, v, w.d[k]);
    }
    const double iv2 = iv * iv, iv4 = iv2 * iv2, iv5 = iv4 * iv, iv8 = iv4 * iv4;
    const double psi_pn = fma(P, iv5, lnv * fma(w.cl6, v, w.cl5));
    const double dpsi = fma(Q, iv8, lnv * w.dl6 * iv2);
    const double dt = (dpsi - w.dpsi_max) * kInvTwoPi;
    const double t = w.tref + dt;
    if (!(f <= w.fcut) || t < 0.0 || t > t_obs) return false;
    // orbit angle alpha(t) = alpha(t_ref) + da
    const float da = (float)(dt * (kTwoPi / kYear));
    float sh, ch;
    sincosf(0.5f * da, &sh, &ch);
    const float sd = 2.0f * sh * ch, omc = 2.0f * sh * sh;   // sin da, 1 - cos da
    const double sa_d = w.sa_ref + (double)(wf.ca_ref * sd - wf.sa_ref * omc);
    const double ca_d = w.ca_ref - (double)(wf.ca_ref * omc + wf.sa_ref * sd);
    const double kc = kAUSec * (w.k[0] * ca_d + w.k[1] * sa_d);
    Phi = kTwoPi * f * (w.tref + kc) + (psi_pn - w.psi_max) - (f - w.fmax) * w.dpsi_max;
    sa = (float)sa_d;
    ca = (float)ca_d;
    const float ivf = (float)iv, ff = (float)f;
    amp = wf.amp * ivf * ivf * ivf * sqrtf(ivf) * expf(-ff * ff * wf.inv_fc2);
    return true;
}

// phase modulo 2 pi in float64, then float32
__device__ __forceinline__ float reduce_phase(double p)
{
    return (float)fma(-rint(p * kInvTwoPi), kTwoPi, p);
}

// Mixed template at f: h = amp e^{-i Phi} T (float32 result).
__device__ __forceinline__ bool point_mixed(const Walker& w, const WalkerF& wf, double f, double f3,
                                            double fm3, double lnf3, double t_obs, float scale,
                                            cf h[3])
{
    double Phi;
    float sa, ca, amp;
    if (!phase_mixed(w, wf, f, f3, fm3, lnf3, t_obs, Phi, sa, ca, amp)) return false;
    float sp, cp;
    sincosf(reduce_phase(Phi), &sp, &cp);
    cf T[3];
    transfer_f32(wf, (float)f, sa, ca, T);
    const cf e = {amp * scale * cp, -amp * scale * sp};
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = fmul(e, T[c]);
    return true;
}

// frequency tables (float64): f^{1/3}, f^{-1/3}, ln(f)/3
__device__ __forceinline__ void freq_tables(double f, double& f3, double& fm3, double& lnf3)
{
    f3 = cbrt(f);
    fm3 = 1.0 / f3;
    lnf3 = log(f) * (1.0 / 3.0);
}

}  // namespace mbh

// ------------------------------------------------------------------------------------------
// templates (complex64 storage)
// ------------------------------------------------------------------------------------------
constexpr int kTplThreadsM = 128;
constexpr int kTplPerThreadM = 4;

__global__ void __launch_bounds__(kTplThreadsM)
    template_mixed_kernel(const double* __restrict__ theta, int64_t W, double f0, double df,
                          int64_t n, double t_obs, float2* __restrict__ h)
{
    __shared__ Walker ws;
    __shared__ WalkerF wsf;
    for (int64_t wi = blockIdx.y; wi < W; wi += gridDim.y) {
        __syncthreads();
        if (threadIdx.x == 0) {
            walker_setup(theta, W, wi, ws);
            walker_f32(ws, wsf);
        }
        __syncthreads();
        const int64_t base = (int64_t)blockIdx.x * kTplThreadsM * kTplPerThreadM + threadIdx.x;
#pragma unroll
        for (int j = 0; j < kTplPerThreadM; ++j) {
            const int64_t k = base + (int64_t)j * kTplThreadsM;
            if (k < n) {
                const double f = f0 + (double)k * df;
                double f3, fm3, lnf3;
                freq_tables(f, f3, fm3, lnf3);
                cf v[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                point_mixed(ws, wsf, f, f3, fm3, lnf3, t_obs, 1.0f, v);
#pragma unroll
                for (int c = 0; c < 3; ++c) h[((int64_t)wi * 3 + c) * n + k] = make_float2(v[c].re, v[c].im);
            }
        }
    }
}

mbh_status mbh::launch_template_mixed(const mbh_grid* g, const double* theta, int64_t W, float2* h,
                                      cudaStream_t st)
{
    const int64_t per_block = (int64_t)kTplThreadsM * kTplPerThreadM;
    dim3 grid((unsigned)((g->n + per_block - 1) / per_block), (unsigned)std::min<int64_t>(W, 65535));
    template_mixed_kernel<<<grid, kTplThreadsM, 0, st>>>(theta, W, g->f0, g->df, g->n, g->t_obs, h);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "template_mixed_kernel");
}

// ------------------------------------------------------------------------------------------
// direct likelihood, fused, mixed precision
// ------------------------------------------------------------------------------------------
constexpr int kDirThreadsM = 256;

// block (walker tile of T, frequency chunk).  The frequency tables and the float32 data of a
// grid point are computed/loaded once and reused by the T walkers.  Data and templates are in
// units where h/sigma is O(1) (float32 range); per-point products are float32, sums float64.
template <int T>
__global__ void __launch_bounds__(kDirThreadsM)
    direct_fused_mixed_kernel(const double* __restrict__ theta, int64_t W, double f0, double df,
                              double t_obs, const float2* __restrict__ wd, const float* __restrict__ wv,
                              int64_t n, int64_t chunk, int nchunks, float inv_sigma,
                              double2* __restrict__ part)
{
    __shared__ Walker ws[T];
    __shared__ WalkerF wsf[T];
    __shared__ double sm[32 * 2 * T];
    const int64_t w0 = (int64_t)blockIdx.x * T;
    const int ch = blockIdx.y;
    if (threadIdx.x < T && w0 + threadIdx.x < W) {
        walker_setup(theta, W, w0 + threadIdx.x, ws[threadIdx.x]);
        walker_f32(ws[threadIdx.x], wsf[threadIdx.x]);
    }
    __syncthreads();
    const int64_t kb = (int64_t)ch * chunk, ke = std::min<int64_t>(n, kb + chunk);
    double acc[2 * T];
#pragma unroll
    for (int t = 0; t < 2 * T; ++t) acc[t] = 0.0;
    for (int64_t k = kb + threadIdx.x; k < ke; k += kDirThreadsM) {
        const double f = f0 + (double)k * df;
        double f3, fm3, lnf3;
        freq_tables(f, f3, fm3, lnf3);
        float2 d[3];
        float v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            d[c] = __ldg(wd + (int64_t)c * n + k);
            v[c] = __ldg(wv + (int64_t)c * n + k);
        }
        for (int t = 0; t < T; ++t) {
            if (w0 + t < W) {
                cf h[3];
                if (point_mixed(ws[t], wsf[t], f, f3, fm3, lnf3, t_obs, inv_sigma, h)) {
                    float pd = 0.0f, ph = 0.0f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        pd += d[c].x * h[c].re + d[c].y * h[c].im;
                        ph += v[c] * (h[c].re * h[c].re + h[c].im * h[c].im);
                    }
                    acc[2 * t] += (double)pd;
                    acc[2 * t + 1] += (double)ph;
                }
            }
        }
    }
    block_sum<2 * T>(acc, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (w0 + t < W) part[(w0 + t) * nchunks + ch] = make_double2(acc[2 * t], acc[2 * t + 1]);
}

mbh_status mbh::launch_direct_fused_mixed(const mbh_data* data, const double* theta, int64_t W,
                                          double* out, cudaStream_t st)
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
    direct_fused_mixed_kernel<T><<<grid, kDirThreadsM, 0, st>>>(
        theta, W, data->grid.f0, data->grid.df, data->grid.t_obs, data->wd32, data->wv32,
        data->grid.n, chunk, nchunks, (float)(1.0 / data->sigma), part);
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
    if (e == cudaSuccess) e = cudaMalloc(&R->mix_sums, sizeof(double) * 2);
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
}

// Edge records of the reference, using the same mixed-precision functions as the walkers so
// that a walker equal to the reference gets dPhi = 0 and rho = 1 up to one rounding.
__global__ void edge_mixed_kernel(const double* __restrict__ theta0, double t_obs,
                                  const double* __restrict__ fe, int n_edges, MixEdge* __restrict__ out)
{
    __shared__ Walker w;
    __shared__ WalkerF wf;
    if (threadIdx.x == 0) {
        walker_setup(theta0, 1, 0, w);
        walker_f32(w, wf);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n_edges; e += blockDim.x) {
        MixEdge m;
        m.f = fe[e];
        freq_tables(m.f, m.f3, m.fm3, m.lnf3);
        double Phi = 0.0;
        float sa, ca, amp;
        m.phi0 = 0.0;
        bool in = phase_mixed(w, wf, m.f, m.f3, m.fm3, m.lnf3, t_obs, Phi, sa, ca, amp);
        cf T[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (in) {
            m.phi0 = Phi;
            transfer_f32(wf, (float)m.f, sa, ca, T);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // 1/H0 in float64: |H0| is ~1e-20..1e-30 in strain units, so |H0|^2 underflows
            // float32, while 1/H0 itself (~1e20..1e30) is a normal float32
            const cf H = fscale(T[c], in ? amp : 0.0f);
            const double hr = (double)H.re, hi = (double)H.im;
            const double m2 = hr * hr + hi * hi;
            m.h0inv[c] = m2 > 0.0 ? make_float2((float)(hr / m2), (float)(-hi / m2)) : make_float2(0.f, 0.f);
        }
        out[e] = m;
    }
}

__global__ void bin_mixed_kernel(const double* __restrict__ summary, const double* __restrict__ invw,
                                 int E, MixBin* __restrict__ out, double* __restrict__ sums)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < E) {
        MixBin m;
#pragma unroll
        for (int j = 0; j < 18; ++j) m.q[j] = (float)summary[(int64_t)b * 18 + j];
        m.invw = (float)invw[b];
        m.pad = 0.0f;
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
    edge_mixed_kernel<<<1, 256, 0, st>>>(R->theta0_dev, R->grid.t_obs, R->fe, E + 1, R->mix_edge);
    bin_mixed_kernel<<<(E + 127) / 128, 128, 0, st>>>(R->summary, R->invw, E, R->mix_bin, R->mix_sums);
    cudaError_t e = cudaGetLastError();
    double sums[2];
    if (e == cudaSuccess) e = cudaMemcpyAsync(sums, R->mix_sums, sizeof sums, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        R->mix.edge = R->mix_edge;
        R->mix.bin = R->mix_bin;
        R->mix.sumA0 = sums[0];
        R->mix.sumB0 = sums[1];
    }
    return e;
}

// ------------------------------------------------------------------------------------------
// heterodyne likelihood, mixed precision
// ------------------------------------------------------------------------------------------
template <int G, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    het_mixed_kernel(const __grid_constant__ HetLaunch L)
{
    constexpr int WPB = BLOCK / G;
    __shared__ Walker ws[WPB];
    __shared__ WalkerF wsf[WPB];
    const int lw = threadIdx.x / G, lane = threadIdx.x % G;
    for (int tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
        int s = 0;
        while (s + 1 < L.n_src && L.src[s + 1].tile_begin <= tile) ++s;
        const SrcDesc& S = L.src[s];
        const int64_t wi = S.w_begin + (int64_t)(tile - S.tile_begin) * WPB + lw;
        const bool active = wi < S.w_end;
        __syncthreads();
        if (lane == 0 && active) {
            walker_setup(L.theta, L.W, wi, ws[lw]);
            walker_f32(ws[lw], wsf[lw]);
        }
        __syncthreads();
        const int E = S.E;
        double adh = 0.0, ahh = 0.0;
        cf carry[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        const int rounds = (E + 1 + G - 1) / G;
        for (int r = 0; r < rounds; ++r) {
            const int e = r * G + lane;
            cf dl[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            if (active && e <= E) {
                const MixEdge me = S.mix.edge[e];
                double Phi;
                float sa, ca, amp;
                if (phase_mixed(ws[lw], wsf[lw], me.f, me.f3, me.fm3, me.lnf3, S.t_obs, Phi, sa, ca, amp)) {
                    float sh, ch;
                    sincosf(0.5f * reduce_phase(Phi - me.phi0), &sh, &ch);
                    const cf em1 = {-2.0f * sh * sh, -2.0f * sh * ch};   // e^{-i dPhi} - 1
                    cf T[3];
                    transfer_f32(wsf[lw], (float)me.f, sa, ca, T);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const cf rho = fmul(fscale(T[c], amp), {me.h0inv[c].x, me.h0inv[c].y});
                        const cf rm1 = {rho.re - 1.0f, rho.im};
                        dl[c] = fadd(fadd(rm1, fmul(rm1, em1)), em1);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) dl[c] = {-1.0f, 0.0f};   // h = 0: r = 0
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
                const MixBin& mb = S.mix.bin[e - 1];
                const float iw = mb.invw;
                float bd = 0.0f, bh = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float d0r = 0.5f * (dp[c].re + dl[c].re), d0i = 0.5f * (dp[c].im + dl[c].im);
                    const float d1r = (dl[c].re - dp[c].re) * iw, d1i = (dl[c].im - dp[c].im) * iw;
                    const float* q = mb.q + 6 * c;
                    bd += q[0] * d0r + q[1] * d0i + q[2] * d1r + q[3] * d1i;
                    bh += q[4] * (2.0f * d0r + d0r * d0r + d0i * d0i) +
                          2.0f * q[5] * (d1r + d0r * d1r + d0i * d1i);
                }
                adh += (double)bd;
                ahh += (double)bh;
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            adh += __shfl_down_sync(0xffffffffu, adh, o, G);
            ahh += __shfl_down_sync(0xffffffffu, ahh, o, G);
        }
        if (active && lane == 0) {
            const double dh = 4.0 * (S.mix.sumA0 + adh);
            const double hh = 4.0 * (S.mix.sumB0 + ahh);
            L.out[wi] = -0.5 * (S.dd + hh - 2.0 * dh);
            L.out[L.W + wi] = dh;
            L.out[2 * L.W + wi] = hh;
        }
    }
}

namespace {
template <int G, int BLOCK>
cudaError_t launch_het_mixed(const HetLaunch& L, int grid, cudaStream_t st)
{
    het_mixed_kernel<G, BLOCK><<<grid, BLOCK, 0, st>>>(L);
    return cudaGetLastError();
}

using HetFn = cudaError_t (*)(const HetLaunch&, int, cudaStream_t);

HetFn pick(int G, int block)
{
#define MBH_CASE(g, b) \
    if (G == g && block == b) return &launch_het_mixed<g, b>;
    MBH_CASE(1, 64) MBH_CASE(1, 128) MBH_CASE(1, 256)
    MBH_CASE(2, 64) MBH_CASE(2, 128) MBH_CASE(2, 256)
    MBH_CASE(4, 64) MBH_CASE(4, 128) MBH_CASE(4, 256)
    MBH_CASE(8, 64) MBH_CASE(8, 128) MBH_CASE(8, 256)
    MBH_CASE(16, 64) MBH_CASE(16, 128) MBH_CASE(16, 256)
    MBH_CASE(32, 64) MBH_CASE(32, 128) MBH_CASE(32, 256)
#undef MBH_CASE
    return nullptr;
}
}  // namespace

mbh_status mbh::run_het_mixed(const mbh_ref* const* refs, const int64_t* offsets, int32_t n_src,
                              const double* theta, int64_t W, double* out, cudaStream_t st,
                              const HetTuning* tuning)
{
    HetTuning t = tuning ? *tuning : HetTuning{8, 128, 0};
    HetFn fn = pick(t.threads_per_walker, t.block);
    if (!fn) return fail(MBH_EINVAL, "unsupported tuning G=%d block=%d", t.threads_per_walker, t.block);
    const int wpb = t.block / t.threads_per_walker;
    static HetLaunch L;
    std::lock_guard<std::mutex> lk(launch_mutex());
    for (int32_t first = 0; first < n_src; first += kMaxSrc) {
        const int32_t count = std::min<int32_t>(kMaxSrc, n_src - first);
        if (mbh_status s = build_launch(refs, offsets, n_src, first, count, wpb, theta, W, out, L)) return s;
        if (L.n_tiles == 0) continue;
        const int grid = t.persistent_blocks > 0 ? std::min(L.n_tiles, t.persistent_blocks) : L.n_tiles;
        cudaError_t e = fn(L, grid, st);
        if (e != cudaSuccess) return cuda_fail(e, "het_mixed_kernel");
    }
    return MBH_OK;
}

// Internal types shared by the translation units of libmbhlike (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/mbhlike.h"

namespace mbh {

constexpr int kMaxBins = 4096;
constexpr int kMaxSrc = 96;   // sources per launch (descriptors travel as kernel parameters)
// default heterodyne blocks (mbh_het_config.block = 0): 224 threads for the mixed (2,2) kernels
// on large batches (the register-capped kernels, 28 resident warps per SM), 128 otherwise
constexpr int kDefaultBlockMixed = 224;
constexpr int kDefaultBlock = 128;

// Edge record of the mixed-precision heterodyne: the frequency tables that make the
// double-float phase chain free of cbrt/log (f, f^{1/3}, f^{-1/3}, ln f / 3 as float pairs),
// the reference's large phase Phi0 (float pair) and 1/H0 of the float32 transfer part
// (h0 = H0 e^{-i Phi0}).
struct MixEdge {
    float2 f, f3, fm3, lnf3, phi0;
    float2 h0inv[3];
    float4 xs;   // sin x, cos x (x = pi f L/c, the one-link phase), 0, x
};
static_assert(sizeof(MixEdge) == 80 && alignof(MixEdge) == 16, "edge records are read as five float4");
// Bin record of the mixed-precision heterodyne: float32 summary data per channel with the
// contraction's factors folded in (q0/2, q1/2, q2/w, q3/w, q4/4, q5/w; w = f_hi - f_lo).
struct alignas(16) MixBin {   // 80 bytes, 16-byte aligned: five 128-bit loads per bin
    float q[18];
    float pad[2];
};
static_assert(sizeof(MixBin) == 80 && alignof(MixBin) == 16, "bin records are read as five float4");

// per (edge, mode) of a higher-mode reference: Phi0_lm (float pair), u = h0_lm/h0 and
// g = e^{-i Phi0_lm}/h0 per channel (float32 complex)
struct MixModeHM {
    float2 phi0;
    float2 u[3];
    float2 g[3];
};

// Extended-precision (double-float) heterodyne tables (mbh_hetx.cu).
// float64 quantities of one parameter vector (Sec. II A), the same derivation for the reference
// and the walkers: PN phase and time coefficients, pinning, cut and taper, amplitude factors, the
// in-plane propagation components (times 2 pi AU/c) and the response constants.
struct XDer {
    double mt, eta, dist;
    double c[8], cl5, cl6;   // Psi_PN = sum_k c_k v^{k-5} + ln v (cl5 + cl6 v); c[5] holds the pinning constant
    double d[8], dl6;        // t(f) = sum_k d_k v^{k-8} + dl6 v^{-2} ln v + t0
    double t0, c1;           // t0 = t_ref - psi'(f_max)/2 pi; c1 = 2 pi t_ref - psi'(f_max)
    double fcut, ifc2;       // f_cut; 1/f_c^2
    double kx, ky;           // 2 pi AU/c (k_x, k_y)
    double k3[3], eu[2], ev[3], G[4];   // k/sqrt3, u/sqrt3, v/sqrt3; mode factors Ga, Gb (re, im)
};
// Edge record (8 x 128-bit loads): f, v0, 1/v0, ln v0, t0(f), cos alpha0, sin alpha0, x, sin 2x,
// cos 2x as float pairs; G_c = K_c/T0_c (complex float pairs) per channel.
struct alignas(16) XEdge {
    float v[32];
};
// Edge weights (8 x 128-bit loads): per channel (war, wai), (wbr, wq) as float pairs; then the
// cross-term weights wc of the three channels; v[30] = 1 where the edge takes the float32 ratio.
struct alignas(16) XWeight {
    float v[32];
};
// Per (edge, mode group) record of a higher-mode reference (5 x 128-bit loads): the group's
// t0(f2) and orbit angle (cos, sin) as float pairs, and per channel G_gc = A0(f2) e^{-i Phi0_g}
// K_c / h0_c (complex float pairs), 0 where h0 = 0; group g = 0..3 holds m = 2, 3, 4, 1.
struct alignas(16) XGrp {
    float v[20];
};

struct MixTables {
    const MixEdge* edge;   // [E+1]
    const MixBin* bin;     // [E]
    double sumA0;          // sum_b sum_c Re A0
    double sumB0;          // sum_b sum_c B0
    const MixModeHM* hm;   // [E+1][6] (higher-mode references)
    const float2* hm_base;  // [E+1][3]: -1 where h0 = 0, else sum u - 1 of the stored u
    double amp_eps0;       // relative rounding of the reference's float32 amplitude factor
    const XDer* xder;      // extended precision: the reference's float64 constants
    const XEdge* xedge;    // [E+1]
    const XWeight* xw;     // [E+1]
    const XGrp* xgrp;      // [E+1][4] higher-mode references
    double xsumA, xsumB;   // 4 sum Re A0, 4 sum B0
    int32_t xn32;          // edges that take the float32 ratio (flagged in their XWeight)
};

// Device-side status word (one per device): the first failed in-kernel check records what
// failed and where; mbh_sync_status reads and clears it.  Kernels only check indices in builds
// with MBH_DEBUG_CHECKS (libmbhlike_debug.so): a failed check records the index and skips the
// access, so a wrong index can never fault or trap.
struct DevStatus {
    unsigned int code;     // 0 = no failure; kDevBounds
    unsigned int kernel;   // kKern*
    int32_t source, pad;   // source (launch slot) of the failing item
    long long index, limit;   // the index and its logical range [0, limit)
};
enum : unsigned int { kDevBounds = 1u };
enum : unsigned int { kKernHetX = 1u, kKernHetF32 = 2u, kKernHetF64 = 3u };
DevStatus* dev_status();   // device address of the current device's status word

#ifdef MBH_DEBUG_CHECKS
__device__ __forceinline__ bool dbg_in_range(DevStatus* st, long long i, long long limit, unsigned kernel,
                                             int src)
{
    if (i >= 0 && i < limit) return true;
    if (st != nullptr && atomicCAS(&st->code, 0u, kDevBounds) == 0u) {
        st->kernel = kernel;
        st->source = src;
        st->index = i;
        st->limit = limit;
    }
    return false;
}
#define MBH_IN_RANGE(st, i, limit, kernel, src) mbh::dbg_in_range((st), (i), (limit), (kernel), (src))
#else
#define MBH_IN_RANGE(st, i, limit, kernel, src) true
#endif

struct PrepItem {
    int32_t bin;
    int64_t k0, k1;   // grid range [k0, k1)
};

struct SrcDesc {
    const double* summary;   // [E][3][6]
    const double2* h0inv;    // [E+1][3]
    const double* fe;        // [E+1]
    const double* invw;      // [E]
    MixTables mix;
    double dd, t_obs;
    float tob_hi, tob_lo;    // t_obs as a float pair (split on the host: no float64 work per edge)
    int64_t w_begin, w_end;  // walker range in theta/out
    int32_t E;
    int32_t E_check;         // logical edge range checked in debug builds: edges [0, E_check]
    int32_t tile_begin;      // first tile of this source
    uint32_t modes;          // mode mask of the reference (1 = (2,2) only)
};

struct HetLaunch {
    const double* theta;
    double* out;
    const void* pt;          // fused sampler half step: the sampler's device state (else null)
    DevStatus* status;       // device status word (in-kernel checks of debug builds)
    int32_t pt_half;
    int64_t W;
    int32_t n_src;
    int32_t n_tiles;
    SrcDesc src[kMaxSrc];
};

mbh_status fail(mbh_status s, const char* fmt, ...);
mbh_status cuda_fail(cudaError_t e, const char* where);
mbh_status check_grid(const mbh_grid* g);
mbh_status check_device();
int sm_count();   // multiprocessors of the current device (148 on B300; cached per device)
mbh_status check_modes(uint32_t modes, mbh_precision precision);
void direct_chunks(int64_t n, int64_t tiles, int64_t max_chunk, int64_t& chunk, int& nchunks,
                   int blocks_per_sm = 32);
mbh_status direct_finish(double2* part, int nchunks, int64_t W, double dd, double* out,
                         cudaStream_t st);
mbh_status launch_direct_finalize(const double2* part, int nchunks, int64_t W, double dd, double* out,
                                  cudaStream_t st);
mbh_status stored_plan(const mbh_data* data, int64_t W, int64_t& chunk, int& nchunks);
mbh_status launch_stored(const mbh_data* data, const void* h, int64_t W, mbh_precision p,
                         double2* part, int64_t chunk, int nchunks, cudaStream_t st);

// mixed-precision entry points (mbh_mixed.cu)
mbh_status launch_template_mixed(const mbh_grid* g, const double* theta, int64_t W, float2* h,
                                 cudaStream_t st, uint32_t modes = 1u);
mbh_status launch_direct_fused_mixed(const mbh_data* data, const double* theta, int64_t W,
                                     double* out, cudaStream_t st, uint32_t modes = 1u);
cudaError_t alloc_ref_tables(mbh_ref* R);
mbh_status make_freq_tables(mbh_data* D, cudaStream_t st);
mbh_status make_x_direct_tables(mbh_data* D, cudaStream_t st);
mbh_status launch_direct_fused_x(const mbh_data* data, const double* theta, int64_t W, double* out,
                                 cudaStream_t st, uint32_t modes = 1u);
void free_ref_tables(mbh_ref* R);
cudaError_t prepare_mixed_tables(mbh_ref* R, cudaStream_t st);
// heterodyne kernel instantiations: launcher and kernel address (for occupancy queries)
using HetLauncher = cudaError_t (*)(const HetLaunch&, int, cudaStream_t);
struct HetKernel {
    HetLauncher launch;
    const void* fn;
};
HetKernel het_kernel_f64(int G, int block);
HetKernel het_kernel_mixed(int G, int block);
HetKernel het_kernel_mixed_hm(int G, int block);
HetKernel het_kernel_mixed_pt(int G, int block);
HetKernel het_kernel_x(int G, int block);
HetKernel het_kernel_x_pt(int G, int block);
mbh_status selftest_df(int kind, const float* x, const float* y, int64_t n, float* o1, float* o2,
                       cudaStream_t st);   // mbh_selftest_math kinds 5, 6
HetKernel het_kernel_xhm(int G, int block);
cudaError_t prepare_x_tables(mbh_ref* R, cudaStream_t st);
cudaError_t prepare_x_tables_hm(mbh_ref* R, cudaStream_t st);
void free_x_tables(mbh_ref* R);
mbh_status het_launch_fused_pt(const mbh_ref* const* refs, int n_ens, int64_t M, const mbh_het_config& cfg,
                               mbh_precision prec, const void* pt_dev, int half, cudaStream_t st);
int fused_pt_block(mbh_precision prec, int G, int64_t M);   // 0: no fused kernel for this shape

// ------------------------------------------------------------------------------------------
// reductions
// ------------------------------------------------------------------------------------------
// Block-wide sum of N doubles per thread; result valid in thread 0.  blockDim.x must be a
// multiple of 32 and <= 1024.  Fixed order.
template <int N>
__device__ void block_sum(double (&v)[N], double* smem /* >= 32*N */)
{
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < N; ++j) smem[j * 32 + warp] = v[j];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double x = lane < nw ? smem[j * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            v[j] = x;
        }
    }
}

}  // namespace mbh

struct mbh_data {
    mbh_grid grid;
    int device = -1;
    double2* wd = nullptr;   // [3][n] 4 df d/S
    double* wv = nullptr;    // [3][n] 4 df/S
    float2* wd32 = nullptr;  // [3][n] sigma 4 df d/S (mixed path)
    float* wv32 = nullptr;   // [3][n] sigma^2 4 df/S (mixed path)
    float4* wsp = nullptr;   // [3][n] float pairs of 2^shift 4 df d/S: (re hi, im hi, re lo, im lo)
    float2* vsp = nullptr;   // [3][n] float pair of 2^(2 shift) 4 df/S
    float4* ftab = nullptr;  // [n] (f hi, f lo, f^{1/3} hi, f^{1/3} lo) of the grid
    float4* ftab2 = nullptr; // [n] (f^{-1/3} hi, lo, ln(f)/3 hi, lo)
    float4* ftab3 = nullptr; // [n] (sin x, cos x, 0, x), x = pi f L/c (the one-link phase)
    float2* wdk = nullptr;   // [3][n] conj(K_c) sigma 4 df d/S: the fused mixed pass's data, with the
    float* wvk = nullptr;    // [3][n] |K_c|^2 sigma^2 4 df/S  frequency-only factors K_c folded in
    float4* ftx = nullptr;   // [n] (x hi, x lo, sin 2x hi, lo), x = pi f L/c: the extended direct pass
    float2* ftx2 = nullptr;  // [n] (cos 2x hi, lo)
    float4* wdx = nullptr;   // [3][n] conj(K_c) sigma 4 df d/S as (re hi, re lo, im hi, im lo)
    float2* wvx = nullptr;   // [3][n] |K_c|^2 sigma^2 4 df/S as a float pair
    double sigma = 1.0;      // scale of the float32 copies: h/sigma is O(1)
    int shift = 0;           // round(log2 sigma): templates are split as h 2^-shift
    double dd = 0.0;         // <d|d>
};

struct mbh_ref {
    int device = -1;
    uint32_t modes = 1u;             // harmonics of h0 and of the walkers' templates
    mbh_grid grid;
    int32_t E = 0;
    int32_t E_check = -1;            // debug builds: logical edge limit of the in-kernel checks (-1: E)
    int64_t band[2] = {0, 0};
    double theta0[11];
    double dd = 0.0;
    std::vector<int64_t> edges_host;
    double* theta0_dev = nullptr;
    int64_t* edges = nullptr;      // [E+1]
    double* fe = nullptr;          // [E+1]
    double* invw = nullptr;        // [E]
    double* summary = nullptr;     // [E][3][6]
    double2* h0e = nullptr;        // [E+1][3]
    double2* h0inv = nullptr;      // [E+1][3]
    mbh::MixEdge* mix_edge = nullptr;
    mbh::MixBin* mix_bin = nullptr;
    double* mix_sums = nullptr;    // device [2]
    mbh::MixModeHM* mix_hm = nullptr;   // higher-mode references: [E+1][6]
    float2* mix_hm_base = nullptr;      // [E+1][3]
    mbh::XDer* x_der = nullptr;         // extended-precision tables ((2,2) references)
    mbh::XEdge* x_edge = nullptr;
    mbh::XWeight* x_w = nullptr;
    double* x_sums = nullptr;
    double* x_sens = nullptr;           // [E+1] per-edge sensitivity of lnL to delta
    mbh::XGrp* x_grp = nullptr;         // higher-mode references: [E+1][4]
    mbh::MixTables mix{};
};

// Heterodyne launch planning (Katz, arXiv:2111.01064, Sec. II B; the batched evaluations of
// Sec. III B-C): walkers of many sources, each with its own bin count, in one launch.
//
//  - A plan packs up to kMaxSrc source descriptors per launch as __grid_constant__ kernel
//    parameters (no host-to-device copy, so a plan can be captured in a CUDA graph).
//  - Tiles of BLOCK/G walkers of one source; G threads per walker deal the edges round-robin
//    (a round covers G bins of a walker).
//  - Persistent mode: grid = SMs x resident blocks, each block loops over tiles; sources are
//    ordered by bin count (largest first) so that the round-robin tile assignment mixes costs.
//    A walker's result does not depend on the order or on the tile that computes it (for a
//    given G, which fixes the order in which its bins are summed).
//  - mbh_het_autotune times the candidate configurations with CUDA events; mbh_het_graph_*
//    capture a plan once and replay it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cmath>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "mbh_internal.cuh"

using namespace mbh;

namespace {

struct HetPlan {
    std::vector<HetLaunch> launches;   // heap-allocated: each ~13 KB
    std::vector<int> grids;
    std::vector<HetKernel> kernels;    // per launch
};

mbh_status check_cfg(const mbh_het_config& c)
{
    const int g = c.threads_per_walker;
    if (!(g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32))
        return fail(MBH_EINVAL, "threads_per_walker %d not in {1,2,4,8,16,32}", g);
    if (c.block != 0 && (c.block < 32 || c.block > 256 || c.block % 32 != 0 || c.block < g))
        return fail(MBH_EINVAL, "block %d not 0 or a multiple of 32 in [32, 256] (and >= threads_per_walker)",
                    c.block);
    return MBH_OK;
}

mbh_status check_het_args(const mbh_ref* const* refs, const int64_t* offsets, int32_t n_src,
                          const double* theta, double* out)
{
    if (n_src < 0) return fail(MBH_EINVAL, "n_sources < 0");
    if (n_src == 0) return MBH_OK;
    if (!refs || !offsets) return fail(MBH_EINVAL, "NULL refs/offsets");
    if (offsets[0] != 0) return fail(MBH_EINVAL, "offsets[0] must be 0");
    int dev = -1;
    cudaGetDevice(&dev);
    for (int32_t s = 0; s < n_src; ++s) {
        if (!refs[s]) return fail(MBH_EINVAL, "refs[%d] is NULL", s);
        if (offsets[s + 1] < offsets[s]) return fail(MBH_EINVAL, "offsets must be non-decreasing");
        if (refs[s]->device != dev) return fail(MBH_EINVAL, "refs[%d] lives on another device", s);
    }
    if (offsets[n_src] > 0 && (!theta || !out)) return fail(MBH_EINVAL, "NULL theta/out");
    return MBH_OK;
}

// Default block (mbh_het_config.block = 0) of the mixed-precision (2,2) kernels for a launch of
// W walkers: 224 threads (the register-capped kernel, 4 blocks of 7 warps per SM) once its
// tiles fill three quarters of such a wave, else 128 (no register cap; below that the capped
// kernel's spills cost more than its occupancy gains).  4, 8 and 16 threads per walker.
int default_block_mixed(int G, int64_t W)
{
    if (G != 4 && G != 8 && G != 16) return kDefaultBlock;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return kDefaultBlock;
    const int64_t wpb = kDefaultBlockMixed / G;
    const int64_t tiles = (W + wpb - 1) / wpb;
    return 4 * tiles >= 3 * 4 * (int64_t)sms ? kDefaultBlockMixed : kDefaultBlock;
}

// Default block of the extended-precision kernels (128 registers; the (2,2) and the higher-mode
// kernel alike: six modes, 16384 walkers, 1.497 against 1.592 ms at 128): with 4 threads per
// walker 256 threads (64 walkers, two full warps of float64 walker set-up, 2 blocks per SM) once
// its tiles fill one and a half blocks per SM, else 128 (32 walkers, 4 blocks per SM): 16384
// walkers x 257 edges take 0.404 ms against 0.414 ms.  Blocks whose walkers do not fill
// whole warps (64, 96, 160 threads) pay for idle lanes in the float64 set-up.  With 8 or 16
// threads per walker (the sampler's smaller half steps) 256 threads: 8192 walkers 0.260 ms
// against 0.286 ms at 128.
int default_block_x(int G, int64_t W)
{
    if (G == 8 || G == 16) return 256;
    if (G != 4) return kDefaultBlock;
    const int sms = sm_count();
    const int64_t tiles = (W + 63) / 64;
    return 2 * tiles >= 3 * (int64_t)sms ? 256 : kDefaultBlock;
}

mbh_status make_plan(const mbh_ref* const* refs, const int64_t* offsets, int32_t n_src,
                     const double* theta, double* out, mbh_precision prec,
                     const mbh_het_config& cfg, HetPlan& plan)
{
    if (mbh_status s = check_cfg(cfg)) return s;
    if (prec != MBH_FP64 && prec != MBH_MIXED && prec != MBH_MIXED_F32)
        return fail(MBH_EINVAL, "unknown precision %d", (int)prec);
    const int64_t W = offsets[n_src];
    // kernel per source: float64 (any modes); MBH_MIXED (2,2): the extended-precision kernel;
    // MBH_MIXED_F32 (2,2): the float32-ratio kernel; mixed with higher modes: the float32-ratio
    // higher-mode kernel.  A launch holds sources of one kernel; block 0 takes each kernel's
    // default block.
    for (int group = 0; group < 2; ++group) {
        std::vector<int32_t> order;
        for (int32_t s = 0; s < n_src; ++s) {
            const bool hm = prec != MBH_FP64 && refs[s]->modes != 1u;
            if ((group == 1) == hm) order.push_back(s);
        }
        if (order.empty()) continue;
        const bool f32_22 = prec == MBH_MIXED_F32 && group == 0;
        const bool x22 = prec == MBH_MIXED && group == 0;
        const bool xhm = prec == MBH_MIXED && group == 1;
        int64_t wg = 0;
        for (int32_t s : order) wg += offsets[s + 1] - offsets[s];
        const int block = cfg.block ? cfg.block
                          : f32_22  ? default_block_mixed(cfg.threads_per_walker, wg)
                          : x22 || xhm ? default_block_x(cfg.threads_per_walker, wg)
                                    : kDefaultBlock;
        const int wpb = block / cfg.threads_per_walker;
        const HetKernel kernel = prec == MBH_FP64 ? het_kernel_f64(cfg.threads_per_walker, block)
                                 : x22            ? het_kernel_x(cfg.threads_per_walker, block)
                                 : xhm            ? het_kernel_xhm(cfg.threads_per_walker, block)
                                 : f32_22         ? het_kernel_mixed(cfg.threads_per_walker, block)
                                                  : het_kernel_mixed_hm(cfg.threads_per_walker, block);
        if (!kernel.launch) return fail(MBH_EINVAL, "no kernel for this configuration");
        if (cfg.persistent)   // largest bin counts first
            std::stable_sort(order.begin(), order.end(),
                             [&](int32_t a, int32_t b) { return refs[a]->E > refs[b]->E; });
        int resident = 0;
        if (cfg.persistent) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            int per_sm = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel.fn, block, 0);
            if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
            resident = std::max(1, per_sm) * sms;
        }
        const int32_t ng = (int32_t)order.size();
        for (int32_t first = 0; first < ng; first += kMaxSrc) {
            const int32_t count = std::min<int32_t>(kMaxSrc, ng - first);
            plan.launches.emplace_back();
            HetLaunch& L = plan.launches.back();
            std::memset(&L, 0, sizeof L);
            L.theta = theta;
            L.W = W;
            L.out = out;
            L.status = dev_status();
            int64_t tiles = 0;
            int32_t j = 0;
            for (int32_t q = 0; q < count; ++q) {
                const int32_t s = order[first + q];
                const int64_t nw = offsets[s + 1] - offsets[s];
                if (nw == 0) continue;
                const mbh_ref* R = refs[s];
                SrcDesc& S = L.src[j++];
                S.summary = R->summary;
                S.h0inv = R->h0inv;
                S.fe = R->fe;
                S.invw = R->invw;
                S.mix = R->mix;
                S.dd = R->dd;
                S.t_obs = R->grid.t_obs;
                S.tob_hi = (float)S.t_obs;
                S.tob_lo = (float)(S.t_obs - (double)S.tob_hi);
                S.E = R->E;
                S.E_check = R->E_check >= 0 ? R->E_check : R->E;
                S.modes = R->modes;
                S.w_begin = offsets[s];
                S.w_end = offsets[s + 1];
                S.tile_begin = (int32_t)tiles;
                tiles += (nw + wpb - 1) / wpb;
                if (tiles > 0x7fffffff) return fail(MBH_EINVAL, "too many walker tiles");
            }
            L.n_src = j;
            L.n_tiles = (int32_t)tiles;
            if (tiles == 0) {
                plan.launches.pop_back();
                continue;
            }
            plan.kernels.push_back(kernel);
            plan.grids.push_back(cfg.persistent ? (int)std::min<int64_t>(tiles, resident) : (int)tiles);
        }
    }
    return MBH_OK;
}

mbh_status run_plan(const HetPlan& plan, cudaStream_t st)
{
    for (size_t i = 0; i < plan.launches.size(); ++i) {
        cudaError_t e = plan.kernels[i].launch(plan.launches[i], plan.grids[i], st);
        if (e != cudaSuccess) return cuda_fail(e, "heterodyne kernel");
    }
    return MBH_OK;
}

// every kernel kind the batch needs exists for this (threads_per_walker, block)
bool plan_has_kernels(const mbh_ref* const* refs, int32_t n_src, mbh_precision prec, const mbh_het_config& c)
{
    for (int32_t s = 0; s < n_src; ++s) {
        const HetKernel k = prec == MBH_FP64    ? het_kernel_f64(c.threads_per_walker, c.block)
                            : refs[s]->modes != 1u ? (prec == MBH_MIXED ? het_kernel_xhm(c.threads_per_walker, c.block)
                                                                        : het_kernel_mixed_hm(c.threads_per_walker, c.block))
                            : prec == MBH_MIXED    ? het_kernel_x(c.threads_per_walker, c.block)
                                                   : het_kernel_mixed(c.threads_per_walker, c.block);
        if (!k.launch) return false;
    }
    return true;
}

// Default launch: 8 threads per walker; 4 for the extended-precision (MBH_MIXED) kernel, whose
// longer edges amortise the walker setup over fewer lanes (measured 10 % faster at 16384 walkers).
mbh_het_config default_cfg(mbh_precision p)
{
    return mbh_het_config{p == MBH_MIXED ? 4 : 8, 0, 0};
}

}  // namespace

struct mbh_het_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int device = -1;
};

extern "C" mbh_status het_loglike_batch_cfg(const mbh_ref* const* refs, const int64_t* offsets_host,
                                            int32_t n_sources, const double* theta_dev,
                                            mbh_precision precision, const mbh_het_config* cfg,
                                            double* out_dev, void* stream)
{
    if (mbh_status s = check_het_args(refs, offsets_host, n_sources, theta_dev, out_dev)) return s;
    if (n_sources == 0 || offsets_host[n_sources] == 0) return MBH_OK;
    const mbh_het_config c = cfg ? *cfg : default_cfg(precision);
    HetPlan plan;
    if (mbh_status s = make_plan(refs, offsets_host, n_sources, theta_dev, out_dev, precision, c, plan)) return s;
    return run_plan(plan, (cudaStream_t)stream);
}

extern "C" mbh_status het_loglike_batch(const mbh_ref* const* refs, const int64_t* offsets_host,
                                        int32_t n_sources, const double* theta_dev,
                                        mbh_precision precision, double* out_dev, void* stream)
{
    return het_loglike_batch_cfg(refs, offsets_host, n_sources, theta_dev, precision, nullptr, out_dev,
                                 stream);
}

extern "C" mbh_status mbh_het_autotune(const mbh_ref* const* refs, const int64_t* offsets_host,
                                       int32_t n_sources, const double* theta_dev,
                                       mbh_precision precision, double* out_dev, int32_t reps,
                                       void* stream, mbh_het_config* best, double* best_ms)
{
    if (!best) return fail(MBH_EINVAL, "best is NULL");
    if (mbh_status s = check_het_args(refs, offsets_host, n_sources, theta_dev, out_dev)) return s;
    if (n_sources == 0 || offsets_host[n_sources] == 0) {
        *best = default_cfg(precision);
        if (best_ms) *best_ms = 0.0;
        return MBH_OK;
    }
    reps = std::max(1, reps);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune events");
    double best_t = INFINITY;
    mbh_het_config best_c = default_cfg(precision);
    const int gs[] = {1, 2, 4, 8, 16, 32};
    const int bs[] = {32, 64, 96, 128, 160, 224, 256};
    mbh_status status = MBH_OK;
    for (int g : gs)
        for (int b : bs)
            for (int pers = 0; pers < 2 && status == MBH_OK; ++pers) {
                if (b < g) continue;
                const mbh_het_config c{g, b, pers};
                HetPlan plan;
                status = make_plan(refs, offsets_host, n_sources, theta_dev, out_dev, precision, c, plan);
                if (status == MBH_EINVAL && !plan_has_kernels(refs, n_sources, precision, c)) {
                    status = MBH_OK;   // no kernel compiled for this pair: not a candidate
                    break;
                }
                if (status != MBH_OK) break;
                status = run_plan(plan, st);   // warm-up
                if (status != MBH_OK) break;
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps && status == MBH_OK; ++r) status = run_plan(plan, st);
                cudaEventRecord(e1, st);
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    status = cuda_fail(e, "autotune");
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double t = ms / reps;
                if (t < best_t) {
                    best_t = t;
                    best_c = c;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != MBH_OK) return status;
    *best = best_c;
    if (best_ms) *best_ms = best_t;
    return MBH_OK;
}

extern "C" mbh_status mbh_het_graph_create(const mbh_ref* const* refs, const int64_t* offsets_host,
                                           int32_t n_sources, const double* theta_dev,
                                           mbh_precision precision, const mbh_het_config* cfg,
                                           double* out_dev, void* stream, mbh_het_graph** out)
{
    if (!out) return fail(MBH_EINVAL, "out is NULL");
    *out = nullptr;
    if (mbh_status s = check_het_args(refs, offsets_host, n_sources, theta_dev, out_dev)) return s;
    const mbh_het_config c = cfg ? *cfg : default_cfg(precision);
    HetPlan plan;
    if (n_sources > 0)
        if (mbh_status s = make_plan(refs, offsets_host, n_sources, theta_dev, out_dev, precision, c, plan)) return s;
    // capture on a private stream so that the caller's stream is never in capture mode
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "graph stream");
    auto G = std::make_unique<mbh_het_graph>();
    cudaGetDevice(&G->device);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    mbh_status status = MBH_OK;
    if (e == cudaSuccess) {
        status = run_plan(plan, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &G->graph);
        if (status == MBH_OK && e2 != cudaSuccess) status = cuda_fail(e2, "end capture");
    } else {
        status = cuda_fail(e, "begin capture");
    }
    if (status == MBH_OK) {
        e = cudaGraphInstantiate(&G->exec, G->graph, 0);
        if (e != cudaSuccess) status = cuda_fail(e, "graph instantiate");
    }
    cudaStreamDestroy(cs);
    if (status != MBH_OK) {
        if (G->exec) cudaGraphExecDestroy(G->exec);
        if (G->graph) cudaGraphDestroy(G->graph);
        return status;
    }
    (void)stream;
    *out = G.release();
    return MBH_OK;
}

extern "C" mbh_status mbh_het_graph_launch(mbh_het_graph* g, void* stream)
{
    if (!g || !g->exec) return fail(MBH_EINVAL, "graph is NULL");
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? MBH_OK : cuda_fail(e, "graph launch");
}

extern "C" void mbh_het_graph_free(mbh_het_graph* g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

namespace mbh {
// Block of a fused half step: the float32-ratio kernel's default, or for the extended kernel
// (whose proposals take shared memory per walker) 32 walkers per block, at most 256 threads.
int fused_pt_block(mbh_precision prec, int G, int64_t M)
{
    if (prec == MBH_MIXED) return std::min(256, 32 * G);
    return default_block_mixed(G, M);
}

// One fused sampler half step (het_mixed_pt_kernel for MBH_MIXED_F32, het_x_pt_kernel for
// MBH_MIXED) over the moving walkers of n_ens ensembles, M of each, ensemble e against refs[e]
// ((2,2) references): multi-source launches (up to kMaxSrc ensembles each) whose walker
// constants come from the sampler's proposals.
mbh_status het_launch_fused_pt(const mbh_ref* const* refs, int n_ens, int64_t M, const mbh_het_config& cfg,
                               mbh_precision prec, const void* pt_dev, int half, cudaStream_t st)
{
    if (mbh_status s = check_cfg(cfg)) return s;
    const int block = cfg.block ? cfg.block : fused_pt_block(prec, cfg.threads_per_walker, M * n_ens);
    const HetKernel k = prec == MBH_MIXED ? het_kernel_x_pt(cfg.threads_per_walker, block)
                                          : het_kernel_mixed_pt(cfg.threads_per_walker, block);
    if (!k.launch) return fail(MBH_EINVAL, "no kernel for this configuration");
    const int wpb = block / cfg.threads_per_walker;
    std::unique_ptr<HetLaunch> L(new (std::nothrow) HetLaunch);
    if (!L) return fail(MBH_ENOMEM, "host allocation");
    int resident = 0;
    if (cfg.persistent) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, block, 0) == cudaSuccess)
            resident = std::max(1, per_sm) * sms;
    }
    for (int first = 0; first < n_ens; first += kMaxSrc) {
        const int count = std::min(kMaxSrc, n_ens - first);
        std::memset(L.get(), 0, sizeof(HetLaunch));
        L->W = M * n_ens;
        L->pt = pt_dev;
        L->pt_half = half;
        L->status = dev_status();
        int64_t tiles = 0;
        for (int q = 0; q < count; ++q) {
            const mbh_ref* R = refs[first + q];
            SrcDesc& S = L->src[q];
            S.summary = R->summary;
            S.h0inv = R->h0inv;
            S.fe = R->fe;
            S.invw = R->invw;
            S.mix = R->mix;
            S.dd = R->dd;
            S.t_obs = R->grid.t_obs;
            S.tob_hi = (float)S.t_obs;
            S.tob_lo = (float)(S.t_obs - (double)S.tob_hi);
            S.E = R->E;
            S.E_check = R->E_check >= 0 ? R->E_check : R->E;
            S.modes = R->modes;
            S.w_begin = (int64_t)(first + q) * M;
            S.w_end = S.w_begin + M;
            S.tile_begin = (int32_t)tiles;
            tiles += (M + wpb - 1) / wpb;
        }
        if (tiles > 0x7fffffff) return fail(MBH_EINVAL, "too many walker tiles");
        L->n_src = count;
        L->n_tiles = (int32_t)tiles;
        const int grid = resident > 0 ? (int)std::min<int64_t>(tiles, resident) : (int)tiles;
        const cudaError_t e = k.launch(*L, grid, st);
        if (e != cudaSuccess) return cuda_fail(e, "fused sampler half step");
    }
    return MBH_OK;
}
}  // namespace mbh

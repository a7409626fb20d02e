/*
 * mbhlike — batched LISA likelihood for massive-black-hole-binary templates on
 * one NVIDIA B300 (sm_103a).  C ABI of libmbhlike.so.
 *
 * The method is the one of Katz, arXiv:2111.01064, Sec. II: frequency-domain
 * (2,2)-mode templates A(f) e^{-i phi(f)} (Eq. 7) put through the LISA TDI A/E/T
 * response at the SPA time t(f) (Eqs. 8-9), the noise-weighted inner product
 * <a|b> = 4 Re sum_{A,E,T} sum_f a* b / S_n df (Eq. 3), the log-likelihood
 * lnL = -1/2 (<d|d> + <h|h> - 2 <d|h>) (Eq. 2), and the heterodyned
 * (relative-binning) likelihood of Sec. II B (Eqs. 10-19) over log-spaced bins
 * covering the band where the reference template is non-zero (Sec. III B).
 * The amplitude/phase model is the stand-in "W0" (TaylorF2 3.5PN phase with
 * aligned-spin terms, Gaussian-tapered f^{-7/6} amplitude, t_ref and phi_ref
 * pinned at f_max = argmax f^2 A) and the response the stand-in "R0" (rigid
 * equal-arm constellation, one-link kernel, first-generation TDI).
 *
 * Conventions shared by every call
 *  - Parameters theta are float64, structure-of-arrays [11][W]:
 *    M_T (solar masses, detector frame), q = m2/m1 in (0, 1], a1, a2 (aligned
 *    spins), D_L (Gpc), phi_ref, iota, lambda, beta, psi (rad, SSB frame),
 *    t_ref (s, time at f_max).
 *  - Frequency grid f_k = f0 + k df, k in [0, n), f0 > 0; a template is zero
 *    above f_cut = 0.2/M and where its track t(f) leaves [0, t_obs].
 *  - Channels are A, E, T in that order; a complex value is two consecutive
 *    numbers (re, im); "complex128" = 2 x float64, "complex64" = 2 x float32.
 *  - Every *_dev pointer is a device pointer owned by the caller; it must stay
 *    valid until the work queued on `stream` has finished.  Handles (mbh_data,
 *    mbh_ref, mbh_het_graph, mbh_server) are owned by the library and released
 *    only by their *_free call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls queue
 *    work asynchronously and return without synchronising, except where a
 *    call says it synchronises.
 *  - Argument errors are detected on the host before anything is queued and
 *    return MBH_EINVAL; CUDA launch/allocation failures return MBH_ECUDA or
 *    MBH_ENOMEM.  mbh_last_error() gives a message for the calling thread.
 *  - There is no host fallback: without a usable CUDA device every compute
 *    call returns MBH_ECUDA.
 */
#ifndef MBHLIKE_H
#define MBHLIKE_H

#include <stdint.h>

#if defined(__GNUC__)
#define MBH_API __attribute__((visibility("default")))
#else
#define MBH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MBH_OK = 0,
    MBH_EINVAL = 1,   /* bad argument (checked on the host, nothing queued) */
    MBH_ENOMEM = 2,   /* device allocation failed */
    MBH_ECUDA = 3,    /* CUDA error (no device, launch failure, ...) */
    MBH_ETIMEOUT = 4, /* a bounded wait gave up (serving loop) */
    MBH_EBUSY = 5,    /* admission refused: over the memory budget or queue full */
    MBH_ECANCELED = 6, /* request cancelled before it was launched */
    MBH_EDEVICE = 7    /* an in-kernel check failed (debug builds): see mbh_sync_status */
} mbh_status;

typedef enum {
    MBH_FP64 = 0,      /* every step in float64 */
    MBH_MIXED = 1,     /* float32-pipe arithmetic with float64-class results where needed.
                          Templates (template_batch, complex64 out): the large phase Phi (Psi +
                          2 pi f k.c) in double-float (two floats, ~48 bits), t(f) in float32
                          with a rounding bound (double-float near the support bounds),
                          amplitude and response in float32.
                          Direct likelihood, (2,2) mode: every step of the template in
                          double-float (phase, t(f), orbit, response, amplitude, taper) and
                          its products with the data, sums in float64; |dlnL| against float64
                          <= 1e-3 up to SNR ~1000 (<h|h> <= 1e6), beyond it ~1e-11 <h|h> (the
                          ~1e6-rad phase carried to |Phi| 2^-48); with higher modes the same per
                          distinct m (direct_loglike_batch_hm).
                          Heterodyne: every edge value formed relative to the reference in
                          double-float (phase, time and amplitude as differences of
                          per-walker float64 coefficients, the response, the ratio
                          delta = r - 1 and the contraction; with higher modes per group of
                          modes sharing m), except on edges of small contraction weight
                          (mbh_ref_f32_edges), which take the MBH_MIXED_F32 ratio within an
                          error budget of 3e-4 in lnL (5e-4 at most while |delta| <= 16,
                          where a walker's edge keeps the float32 value); |dlnL| against
                          float64 <= 1e-3 up to SNR ~1000. */
    MBH_MIXED_F32 = 2  /* heterodyne: double-float phase difference, float32 response,
                          ratio delta = r - 1 and per-bin products, double-float sums.  About
                          3x faster than MBH_MIXED; its |dlnL| grows with <h|h> (~1e-3 at
                          SNR ~120, beyond it above).  Direct likelihood: the template as
                          template_batch's MBH_MIXED, products with the data in float32 on
                          O(1)-scaled operands, sums in float64 (|dlnL| <= ~1e-5 of
                          (<d|d> + <h|h> + 2|<d|h>|)/2; 3.7x faster than MBH_MIXED). */
} mbh_precision;

typedef struct {
    double f0;     /* first grid frequency (Hz), > 0 */
    double df;     /* spacing (Hz), > 0 */
    int64_t n;     /* number of grid points, >= 2 */
    double t_obs;  /* observation window [0, t_obs] (s) */
} mbh_grid;

typedef struct mbh_data mbh_data; /* data d~ and noise weights on one grid */
typedef struct mbh_ref mbh_ref;   /* one heterodyne reference (summary data) */

/* Message for the last failing call on this thread ("" if none). */
MBH_API const char* mbh_last_error(void);

/* ---- device-side status word -----------------------------------------------------
 * The paper has no counterpart: this is the library's error channel for what only a
 * kernel can see.  Every device holds one status word.  The heterodyne kernels of a build
 * with MBH_DEBUG_CHECKS (libmbhlike_debug.so, built by `python -m
 * paper_2111_01064_b300.build --debug`) check the index of every bin-edge record they read
 * against the reference's logical edge range; the first failed check on a device records
 * the kernel, the source slot, the index and its range, and the kernel skips that access
 * (it never traps, faults or waits).  Release builds do no in-kernel checks.  Calls never
 * read the word on their own (that would synchronise): mbh_sync_status does. */
typedef struct {
    int32_t code;     /* 0: no failure; 1: an index outside its logical range */
    int32_t kernel;   /* 1: MBH_MIXED heterodyne, 2: MBH_MIXED_F32, 3: MBH_FP64 */
    int32_t source;   /* launch slot of the failing walker's source */
    int32_t reserved;
    int64_t index;    /* the failing index and its range [0, limit) */
    int64_t limit;
} mbh_device_status;

/* Synchronises `stream`, then reads and clears the current device's status word.
 * MBH_OK if no check failed; MBH_EDEVICE (details in *info, if not NULL, and in
 * mbh_last_error) if one did; MBH_ECUDA for an asynchronous CUDA error of the stream's
 * work (cudaStreamSynchronize's).  info is zeroed when nothing failed. */
MBH_API mbh_status mbh_sync_status(void* stream, mbh_device_status* info);
/* 1 if this library was built with MBH_DEBUG_CHECKS, else 0. */
MBH_API int32_t mbh_debug_checks(void);

/* Analytic noise PSD S_n of A, E, T on the grid (Sec. II, remark under Eq. 3:
 * A and E identical, T different; acceleration 3e-15 m/s^2/rtHz, OMS
 * 15e-12 m/rtHz, L = 2.5e9 m).  psd_dev: float64 [3][n], written. */
MBH_API mbh_status mbh_psd_aet(const mbh_grid* grid, double* psd_dev, void* stream);

/* Gaussian noise realisation from standard normals (Sec. II: <n~ n~*> = S/2 per
 * unit bandwidth): noise[c][k] = sqrt(S[c][k] / (4 df)) (z[c][k][0] + i z[c][k][1]).
 * z_dev: float64 [3][n][2]; psd_dev: float64 [3][n]; noise_dev: complex128
 * [3][n], written.  With accumulate != 0 the noise is added to noise_dev. */
MBH_API mbh_status mbh_noise_aet(const mbh_grid* grid, const double* z_dev, const double* psd_dev,
                         int32_t accumulate, void* noise_dev, void* stream);

/* Templates h~^{A,E,T}(f_k) = T^{A,E,T}(f, t(f)) A(f) e^{-i phi(f)} on the grid
 * (Sec. II A, Eqs. 7-9).  theta_dev: float64 [11][W]; h_out_dev: [W][3][n]
 * complex128 (MBH_FP64) or complex64 (MBH_MIXED: the float64 phase is rounded
 * once to float32 storage), written. */
MBH_API mbh_status template_batch(const mbh_grid* grid, const double* theta_dev, int64_t W,
                          mbh_precision precision, void* h_out_dev, void* stream);

/* Bind data to a grid (Sec. II, Eq. 3).  d_dev: complex128 [3][n]; psd_dev:
 * float64 [3][n] (all > 0).  The library keeps its own device copies (the
 * caller's buffers may be released once the stream has passed this call) in
 * the form 4 df d/S (complex128) and 4 df/S (float64), and computes <d|d>.
 * Synchronises `stream` once (to read <d|d>). */
MBH_API mbh_status mbh_data_create(const mbh_grid* grid, const void* d_dev, const double* psd_dev,
                           void* stream, mbh_data** out);
/* <d|d> of the data (host value, computed at creation). */
MBH_API double mbh_data_dd(const mbh_data* data);
MBH_API void mbh_data_free(mbh_data* data);

/* Direct likelihood, templates generated on the device and reduced in the same
 * pass (Sec. II, Eqs. 2-3; Sec. III A).  out_dev: float64 [3][W]: lnL, <d|h>,
 * <h|h>.  MBH_MIXED evaluates the template and its products in double-float,
 * MBH_MIXED_F32 the response in float32 around double-float phases; sums are
 * float64 in every mode. */
MBH_API mbh_status direct_loglike_batch(const mbh_data* data, const double* theta_dev, int64_t W,
                                mbh_precision precision, double* out_dev, void* stream);

/* Direct likelihood of stored templates h_dev [W][3][n] (complex128 for
 * MBH_FP64, complex64 for MBH_MIXED), e.g. from template_batch.  Float64
 * accumulation.  out_dev as above. */
MBH_API mbh_status direct_loglike_stored(const mbh_data* data, const void* h_dev, int64_t W,
                                 mbh_precision precision, double* out_dev, void* stream);

/* direct_loglike_stored without device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory while they
 * evaluate likelihoods (a fixed memory budget owned by another framework, a host
 * callback that must not enter the allocator, a service that reserves all device
 * memory up front).  Same arguments, layout and result as direct_loglike_stored; the
 * partial sums live in one static 8 MiB device buffer held by every device that loads
 * the library until the process exits.
 *  - Size limit: W x (number of grid chunks) x 16 bytes must fit in 8 MiB; large
 *    batches use at least n / 262144 chunks, so on a 1,051,920-point grid W can
 *    reach ~100,000 templates.  Larger batches return MBH_EINVAL with the required
 *    size in mbh_last_error(), checked before anything is queued.
 *  - The first call on a device looks up the buffer's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call before
 *    any stream capture.
 *  - All calls on a device share the buffer: calls whose work overlaps on the GPU
 *    (different streams, or different host threads) race and give wrong results;
 *    serialise them, e.g. on one stream.
 *  - Calls no cudaMalloc, cudaFree or other allocating routine. */
MBH_API mbh_status direct_loglike_stored_noalloc(const mbh_data* data, const void* h_dev, int64_t W,
                                         mbh_precision precision, double* out_dev, void* stream);

/* Heterodyne reference (Sec. II B, Eqs. 15-16 and 18-19; Sec. III B).
 * theta0_host: float64 [11] on the host.  Band = first..last grid index where
 * h0 != 0; n_bins + 1 log-spaced edge targets from f(band start) to f(band end)
 * rounded to the nearest grid index, endpoints exact, duplicates dropped.  Bin
 * b holds k in [e_b, e_{b+1}), the last bin also e_E; f_b is the bin centre.
 * Stores per bin and channel A0, A1 (complex), B0, B1 (real), h0 at the edges
 * and <d|d>.  The handle is independent of `data` afterwards.  Synchronises
 * `stream` (edge bookkeeping on the host).  MBH_EINVAL if the band has fewer
 * than two grid points or n_bins is outside [1, 4096]. */
MBH_API mbh_status het_prepare_reference(const mbh_data* data, const double* theta0_host,
                                 int32_t n_bins, void* stream, mbh_ref** out);
/* Number of bins E actually used (<= n_bins). */
MBH_API int32_t mbh_ref_bins(const mbh_ref* ref);
/* Mode mask the reference was prepared with (see the higher-harmonic calls). */
MBH_API uint32_t mbh_ref_modes(const mbh_ref* ref);
/* Edges (of the E + 1) that MBH_MIXED evaluates with the float32 ratio instead of the
 * double-float chain: the per-edge precision choice made at prepare from the contraction
 * weights (Eqs. 14 and 17 regrouped per edge), see MBH_MIXED.  -1 for a NULL reference. */
MBH_API int32_t mbh_ref_f32_edges(const mbh_ref* ref);
/* Copies (host, blocking): edges int64 [E+1]; summary float64 [E][3][6] =
 * Re A0, Im A0, Re A1, Im A1, B0, B1; h0 at the edges complex128 [E+1][3];
 * any pointer may be NULL. */
MBH_API mbh_status mbh_ref_read(const mbh_ref* ref, int64_t* edges_host, double* summary_host,
                        double* h0_edges_host, double* dd_host);
MBH_API void mbh_ref_free(mbh_ref* ref);
/* Test support of debug builds: narrows the logical edge range that the in-kernel checks
 * hold the reference's edge indices to, edges [0, e_check] (-1 restores [0, E]); the
 * tables themselves and the kernels' loops are unchanged, so indices past e_check stay
 * inside the allocated records and the checks, not the memory, decide.  MBH_EINVAL for
 * e_check outside [-1, E], and in release builds (no in-kernel checks). */
MBH_API mbh_status mbh_debug_ref_limit(mbh_ref* ref, int32_t e_check);

/* Heterodyned likelihood for walkers of several sources in one launch
 * (Sec. II B, Eqs. 14 and 17): the template is evaluated at the E_s + 1 bin
 * edges of its source, r = h/h0, r0 = (r_lo + r_hi)/2, r1 = (r_hi - r_lo)/(f_hi -
 * f_lo), and contracted with the summary data.  Walkers [offsets[s],
 * offsets[s+1]) belong to refs[s]; theta_dev: float64 [11][W] with W =
 * offsets[n_sources]; offsets_host: int64 [n_sources + 1] on the host,
 * non-decreasing, offsets[0] = 0.  out_dev: float64 [3][W]: lnL, <d|h>, <h|h>.
 * MBH_MIXED: float64 phase difference, float32 ratios in the delta = r - 1
 * form, float32 products accumulated in float64. */
MBH_API mbh_status het_loglike_batch(const mbh_ref* const* refs, const int64_t* offsets_host,
                             int32_t n_sources, const double* theta_dev,
                             mbh_precision precision, double* out_dev, void* stream);

/* Test support: evaluates the library's own float32 device math on n inputs
 * (float32 device arrays) so that it can be checked against CUDA's functions and
 * float64 references.  kind 0: sin and cos of x (o1, o2; Cody-Waite reduction and
 * Taylor polynomials, |x| up to ~100); kind 1: sin(x)/x (o1); kind 2:
 * sinc(x(1+y)) - sinc(x(1-y)) without cancellation (o1); kinds 3 and 4: the
 * four-term forms of kinds 1 and 2 that the response uses below x = 0.1 (valid for
 * |x| < 0.2, and x < 0.1 with |y| <= 1).  The double-float (two-float) math of the
 * extended-precision kernels, n values as (hi, lo) pairs (x: 2n floats; o1, o2: 2n
 * floats): kind 5: sin and cos - 1 of x (o1, o2; any |x| < 2^22 pi, the pairs need not
 * be normalised); kind 6: x y - n 2 pi with y three floats per value (3n floats, a
 * triple-float), n = round(x.hi y.hi / 2 pi) (o1).  MBH_EINVAL for another kind. */
MBH_API mbh_status mbh_selftest_math(int32_t kind, const float* x_dev, const float* y_dev, int64_t n,
                             float* o1_dev, float* o2_dev, void* stream);

/* Launch configuration of the heterodyne kernels.  A walker is handled by
 * threads_per_walker threads (1, 2, 4, 8, 16 or 32) that deal its bin edges
 * round-robin (each round covers threads_per_walker bins); a block of `block`
 * threads holds block/threads_per_walker walkers of one source.  Every kernel has
 * blocks of 64, 128 and 256 threads; the mixed-precision (2,2) kernels (and the
 * fused sampler half step) also 224 for 4, 8 or 16 threads per walker, 96 and 160
 * for 4 or 8, and 32 for 2 or 4, compiled for ~28 resident warps per SM (72
 * registers); a (threads_per_walker, block) pair without a kernel is rejected
 * (MBH_EINVAL).  block = 0 takes the default: 224 for the mixed (2,2) kernels at 4,
 * 8 or 16 threads per walker when the launch has at least 3 x (SMs) blocks of 224
 * threads' worth of walkers (16384 walkers at 8 threads per walker on 148 SMs),
 * else 128.
 * persistent = 0: one block per walker tile; 1: a grid of (SMs x resident blocks)
 * looping over the tiles, sources ordered by bin count (largest first).  For a
 * given threads_per_walker the results are bitwise reproducible and independent of
 * the block size, the persistent mode, the other walkers and sources in the launch
 * and their order; threads_per_walker sets the order in which a walker's bins are
 * summed, so changing it changes results in the last bits only. */
typedef struct {
    int32_t threads_per_walker;
    int32_t block;
    int32_t persistent;
} mbh_het_config;

/* het_loglike_batch with an explicit launch configuration (NULL = default). */
MBH_API mbh_status het_loglike_batch_cfg(const mbh_ref* const* refs, const int64_t* offsets_host,
                                 int32_t n_sources, const double* theta_dev,
                                 mbh_precision precision, const mbh_het_config* cfg,
                                 double* out_dev, void* stream);

/* Autotuner for a given batch (same arguments as het_loglike_batch): times every
 * configuration (reps launches each after one warm-up, CUDA events on `stream`),
 * writes the fastest to *best and its time per batch to *best_ms.  out_dev is
 * overwritten.  Synchronises `stream`. */
MBH_API mbh_status mbh_het_autotune(const mbh_ref* const* refs, const int64_t* offsets_host,
                            int32_t n_sources, const double* theta_dev, mbh_precision precision,
                            double* out_dev, int32_t reps, void* stream, mbh_het_config* best,
                            double* best_ms);

/* A heterodyne batch captured once in a CUDA graph (on a private stream) and
 * replayed with mbh_het_graph_launch: the refs, offsets, theta_dev and out_dev
 * pointers are fixed at creation; the caller rewrites theta_dev in place between
 * replays (e.g. one sampler step per replay).  The refs must outlive the graph. */
typedef struct mbh_het_graph mbh_het_graph;
MBH_API mbh_status mbh_het_graph_create(const mbh_ref* const* refs, const int64_t* offsets_host,
                                int32_t n_sources, const double* theta_dev, mbh_precision precision,
                                const mbh_het_config* cfg, double* out_dev, void* stream,
                                mbh_het_graph** out);
MBH_API mbh_status mbh_het_graph_launch(mbh_het_graph* graph, void* stream);
MBH_API void mbh_het_graph_free(mbh_het_graph* graph);

/* ---- serving loop --------------------------------------------------------------
 * Continuous batching of heterodyned-likelihood requests from many concurrent
 * samplers (the batched evaluations of Sec. III B-C) on the current device.
 * Sources (prepared references) stay resident on the device and are admitted while
 * their footprint fits hbm_budget_bytes.  A request = one source and W walkers;
 * submit copies theta (the caller may reuse its buffer on return) and queues it; a
 * worker thread packs queued requests of any sources into one multi-source launch
 * whenever one of max_inflight_batches slots (fixed device buffers for
 * max_batch_walkers walkers, counted in the budget, one stream each) is free, so a
 * new batch's copies and kernel overlap those in flight.  A request's results are
 * the same alone and in a batch. */
typedef struct mbh_server mbh_server;
typedef struct {
    int64_t hbm_budget_bytes;       /* device memory for slots + resident sources */
    int32_t max_batch_walkers;      /* walkers per launch (and per request) */
    int32_t max_inflight_batches;   /* slots */
    int32_t max_queue;              /* queued requests before submit returns MBH_EBUSY */
    mbh_precision precision;
    mbh_het_config config;          /* threads_per_walker = 0: default configuration */
} mbh_server_opts;
typedef struct {
    int64_t completed, walkers, batches, rejected, queued;
    double mean_batch_walkers;
    double p50_ms, p99_ms, max_ms;  /* submit -> results written, completed requests */
    double walkers_per_s;           /* walkers completed / (first submit .. last completion) */
    int64_t source_bytes, slot_bytes;
} mbh_server_report;

/* Starts the worker thread.  MBH_EBUSY if the slots alone exceed the budget. */
MBH_API mbh_status mbh_server_create(const mbh_server_opts* opts, mbh_server** out);
/* Registers a prepared reference (which must outlive the server or its removal);
 * MBH_EBUSY if it does not fit the budget. */
MBH_API mbh_status mbh_server_add_source(mbh_server* server, const mbh_ref* ref, int32_t* source_id);
/* Evicts a source: its queued requests complete with MBH_EINVAL, batches in flight
 * finish first (the call blocks until then). */
MBH_API mbh_status mbh_server_remove_source(mbh_server* server, int32_t source_id);
/* Reference refresh (Sec. III B: the reference is replaced by the best walker every
 * few thousand sampler iterations): every request of the source launched after the
 * call uses `ref` (prepared, e.g., around the best walker, with its band re-selected
 * by het_prepare_reference); requests already queued but not launched use it too.
 * Returns once the batches in flight on the previous reference have finished, so the
 * caller may then free it.  MBH_EBUSY if the new reference does not fit the budget. */
MBH_API mbh_status mbh_server_replace_source(mbh_server* server, int32_t source_id, const mbh_ref* ref);
/* theta_host: float64 [11][W]; out_host: float64 [3][W] (lnL, <d|h>, <h|h>), written
 * on completion and owned by the caller until mbh_server_wait returns.  MBH_EBUSY
 * when the queue is full, MBH_EINVAL for an unknown source or W outside
 * [1, max_batch_walkers]. */
MBH_API mbh_status mbh_server_submit(mbh_server* server, int32_t source_id, const double* theta_host,
                             int64_t W, double* out_host, uint64_t* request_id);
/* Waits up to timeout_ms (< 0: no limit); MBH_ETIMEOUT if the request is not done.
 * *request_status: MBH_OK, MBH_ECANCELED, MBH_EINVAL (source evicted) or a CUDA
 * error of its batch.  A request can be waited for once. */
MBH_API mbh_status mbh_server_wait(mbh_server* server, uint64_t request_id, int32_t timeout_ms,
                           mbh_status* request_status);
/* paused != 0: keep admitting and queueing requests but launch nothing (batches
 * already in flight finish); 0: resume. */
MBH_API mbh_status mbh_server_pause(mbh_server* server, int32_t paused);
/* Cancels a request that has not been launched (MBH_EBUSY once it has). */
MBH_API mbh_status mbh_server_cancel(mbh_server* server, uint64_t request_id);
MBH_API mbh_status mbh_server_stats(mbh_server* server, mbh_server_report* out);
MBH_API mbh_status mbh_server_reset_stats(mbh_server* server);
/* Cancels queued requests, waits for batches in flight, stops the worker. */
MBH_API void mbh_server_free(mbh_server* server);

/* Load generator for measuring a server (no counterpart in the paper; the
 * "sampler threads" of a serving benchmark): n_clients threads, client c submits
 * requests for source_ids[c] at Poisson arrival times with total rate
 * rate_per_s for `seconds` (open loop), sizes log-uniform in
 * [min_walkers, max_walkers], walkers copied from pools_host[c] (host float64
 * [11][pool], SoA); results are reaped as they complete.  Resets the server's
 * statistics first; blocks until every accepted request has completed.  Requests
 * refused by a full queue count as rejected.  MBH_EINVAL for bad options (including more
 * than 1e7 arrivals in total). */
typedef struct {
    double rate_per_s;
    double seconds;
    int32_t min_walkers, max_walkers;
    uint64_t seed;
} mbh_loadgen_opts;
typedef struct {
    double offered_per_s;
    int64_t submitted, completed, rejected, failed;
    double wall_seconds, completed_per_s, walkers_per_s;
    double p50_ms, p99_ms, max_ms;        /* submit -> results written, server side */
    int64_t batches;
    double mean_batch_walkers;
} mbh_loadgen_report;
MBH_API mbh_status mbh_server_loadgen(mbh_server* server, const int32_t* source_ids, int32_t n_clients,
                                      const double* const* pools_host, int64_t pool,
                                      const mbh_loadgen_opts* opts, mbh_loadgen_report* out);

/* ---- Higher harmonics (Sec. II A, Eqs. 7-9) ------------------------------
 * Templates summed over harmonic modes (l, m), each with its own time-frequency
 * map t_lm(f) (Eq. 8) and its own response at t_lm (Eq. 9).  The model is the
 * stand-in "W0-HM" (PhenomHM's coefficients are not available): mode (l, m) takes
 * the W0 (2,2) phase at f2 = 2f/m scaled by m/2, so t_lm(f) = t_22(2f/m), and the
 * (2,2) amplitude at f2 times sqrt(2/m) and the leading post-Newtonian mode factor
 * H_lm(x), x = (pi M f2)^{2/3}; polarisations from the spin-weighted harmonics
 * -2Y_lm(iota, phi_ref).  Mode mask: bit 0 (2,2), bit 1 (3,3), bit 2 (4,4),
 * bit 3 (2,1), bit 4 (3,2), bit 5 (4,3); mask 1 is W0 and these calls then do
 * exactly what the (2,2) calls do.  Mixed precisions: templates (complex64) and
 * MBH_MIXED_F32 evaluate each mode's large phase in double-float and its response in
 * float32; MBH_MIXED evaluates the direct likelihood's template and products in
 * double-float, and the heterodyne ratio relative to the reference per group of modes
 * sharing m (as for the (2,2) mode).  Layouts, ownership and errors as in the (2,2)
 * calls; an empty mask or bits above 5 return MBH_EINVAL. */
MBH_API mbh_status template_batch_hm(const mbh_grid* grid, const double* theta_dev, int64_t W,
                                     uint32_t modes, mbh_precision precision, void* h_out_dev,
                                     void* stream);
MBH_API mbh_status direct_loglike_batch_hm(const mbh_data* data, const double* theta_dev, int64_t W,
                                           uint32_t modes, mbh_precision precision, double* out_dev,
                                           void* stream);
/* The band is where some selected mode of h0 is non-zero; het_loglike_batch then
 * evaluates every walker of this reference with the same modes (either precision;
 * a launch mixing (2,2) and higher-mode references runs one kernel per kind). */
MBH_API mbh_status het_prepare_reference_hm(const mbh_data* data, const double* theta0_host,
                                            int32_t n_bins, uint32_t modes, void* stream,
                                            mbh_ref** out);

/* ---- Parallel-tempered ensemble sampler iteration (Sec. III) -------------
 * The sampler shared by the paper's three pipeline modules, run on the device:
 * T temperatures (inverse temperatures beta_t, target L^beta_t x prior) of W
 * walkers.  Walkers move in x = (ln M_T, q, a1, a2, D_L, phi_ref, cos iota,
 * lambda, sin beta, psi, t_ref), whose prior (Table I) is uniform on the box
 * [lo, hi].  One iteration: the two halves of every temperature move in turn,
 * each against the other half (stretch move, Goodman & Weare 2010, with
 * probability probs[0]; otherwise a sky-mode hop of Sec. III: all eight modes
 * (probs[1]), a longitudinal change (probs[2]) or the latitudinal flip
 * (probs[3])), every proposal batch is scored with het_loglike_batch (ref) or
 * direct_loglike_batch (data), tempered Metropolis acceptance; then swaps
 * between adjacent temperatures, hottest pair first, walkers paired by a random
 * permutation (parallel tempering, Vousden, Farr & Mandel 2016).  Random numbers
 * are Philox4x32-10 (Salmon et al. 2011) with key = seed and counter = (item,
 * purpose, iteration): a run is reproducible and independent of launch
 * configuration, and positions are bit-exact functions of (seed, start state)
 * for a given likelihood.  The iteration counter lives on the device, so
 * iterations replay from a CUDA graph without host work.
 *
 * Ownership: the handle owns the ensemble state (device), the scratch and a
 * captured graph; it keeps pointers to ref/data, which must outlive it (or be
 * replaced with mbh_pt_set_ref first).  Counters (int64, 10 T): [0, 4T)
 * proposals per (temperature, kind), [4T, 8T) accepted per (temperature, kind),
 * kinds in the order of probs; [8T, 9T) accepted swaps per level i (pair i,
 * i-1; entry 0 unused); [9T, 10T) proposed swaps per level.
 * Errors: MBH_EINVAL for bad options (T not in [1, 64], W odd or not in
 * [4, 8192], a <= 1, negative probabilities or a sum outside (0, 1], lo > hi,
 * negative or non-finite betas, not exactly one of ref/data). */
typedef struct mbh_pt mbh_pt;
typedef struct {
    int32_t ntemps;          /* T */
    int32_t walkers;         /* W per temperature */
    double a;                /* stretch scale (2 in Goodman & Weare) */
    double probs[4];         /* stretch, all 8 sky modes, longitudinal, latitudinal */
    double lo[11], hi[11];   /* prior box in x */
    uint64_t seed;
    mbh_precision precision;           /* of the likelihood */
    mbh_het_config het_config;         /* threads_per_walker 0 = default: 16 threads per walker
                                          when a half step moves <= 12288 walkers (mixed
                                          precision), else 8; block 0 = default */
    uint32_t modes;                    /* direct likelihood: harmonic mode mask (0 = (2,2));
                                          a reference brings its own */
    double adapt_time;                 /* > 0: adapt the ladder every iteration (Vousden et
                                          al. 2016): ln(T_t - T_{t-1}) moves by kappa (A_t -
                                          A_{t+1}), kappa = n0/(adapt_time (n + n0)), A_t this
                                          iteration's swap acceptance of pair (t, t-1); the
                                          coldest and hottest temperatures stay fixed */
    double adapt_lag;                  /* n0 (> 0 when adapting) */
    int32_t no_fuse;                   /* != 0: keep proposal, likelihood and acceptance as
                                          separate launches (by default a mixed-precision
                                          (2,2) reference runs each half step as one fused
                                          heterodyne launch) */
} mbh_pt_opts;

/* x_dev: float64 [11][T W] start positions in x, slot t W + k = walker k of
 * temperature t (inside the prior box: outside it, cos iota and sin beta are
 * clamped to [-1, 1] for scoring); betas_host: [T].  Scores the start state
 * and synchronises `stream` before returning. */
MBH_API mbh_status mbh_pt_create(const mbh_pt_opts* opts, const mbh_ref* ref, const mbh_data* data,
                                 const double* betas_host, const double* x_dev, void* stream,
                                 mbh_pt** out);
/* Several independent ensembles stepping together (one per source, or independent
 * chains of one source): ensemble e uses refs[e] (or, with data, the direct
 * likelihood of the common data), seed seed + e 0x9E3779B97F4A7C15, ladder
 * betas_host[e T .. e T + T) and slots [e T W, (e+1) T W) of x_dev [11][n_ens T W];
 * it is exactly a single-ensemble sampler with that seed.  A half step of all
 * ensembles is one likelihood batch, which fills the GPU where one ensemble's half
 * step does not.  Counters are [n_ens][10 T].  n_ens in [1, 1024]. */
MBH_API mbh_status mbh_pt_create_multi(const mbh_pt_opts* opts, const mbh_ref* const* refs, int32_t n_ens,
                                       const mbh_data* data, const double* betas_host, const double* x_dev,
                                       void* stream, mbh_pt** out);
/* Queues n_iter iterations on `stream` (use_graph != 0: replays of one
 * captured iteration). */
MBH_API mbh_status mbh_pt_run(mbh_pt* pt, int64_t n_iter, int32_t use_graph, void* stream);
/* Copies the state in slot order: x_dev [11][n_ens T W], out_dev [3][n_ens T W]
 * (lnL, <d|h>, <h|h>); either may be NULL. */
MBH_API mbh_status mbh_pt_state(const mbh_pt* pt, double* x_dev, double* out_dev, void* stream);
/* Replaces the positions (slot order) and rescores them. */
MBH_API mbh_status mbh_pt_set_state(mbh_pt* pt, const double* x_dev, void* stream);
/* Reference refresh (Sec. III B): later iterations use `ref`; every walker is
 * rescored against it (single-ensemble samplers; mbh_pt_set_ref_at for ensemble e). */
MBH_API mbh_status mbh_pt_set_ref(mbh_pt* pt, const mbh_ref* ref, void* stream);
MBH_API mbh_status mbh_pt_set_ref_at(mbh_pt* pt, int32_t ensemble, const mbh_ref* ref, void* stream);
/* Current inverse temperatures [n_ens][T] (after any adaptation; synchronises `stream`). */
MBH_API mbh_status mbh_pt_get_betas(const mbh_pt* pt, double* betas_host, void* stream);
/* New inverse temperatures [n_ens][T] (synchronises `stream`). */
MBH_API mbh_status mbh_pt_set_betas(mbh_pt* pt, const double* betas_host, void* stream);
/* Reads the counters and the iteration counter (synchronises `stream`). */
MBH_API mbh_status mbh_pt_counters(const mbh_pt* pt, int64_t* counters_host, uint64_t* step_host,
                                   void* stream);
/* Walker of temperature `temp` with the largest lnL (lowest slot on ties):
 * x_host [11], out_host [3] (synchronises `stream`). */
MBH_API mbh_status mbh_pt_best(const mbh_pt* pt, int32_t temp, double* x_host, double* out_host,
                               void* stream);
/* The same for ensemble `ensemble`. */
MBH_API mbh_status mbh_pt_best_at(const mbh_pt* pt, int32_t ensemble, int32_t temp, double* x_host,
                                  double* out_host, void* stream);
MBH_API void mbh_pt_free(mbh_pt* pt);

#ifdef __cplusplus
}
#endif
#endif /* MBHLIKE_H */

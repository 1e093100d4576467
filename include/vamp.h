/*
 * vamp.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot
 * path of the doubly adaptive multi-channel Monte-Carlo integrator (VAMP) of
 * arXiv:1811.09711.
 *
 * The library integrates f over the unit hypercube [0,1]^d with K phase-space
 * channels φ_c, each carrying its own adaptive VEGAS grid G_c (§3.2, §3.5):
 *
 *     I = Σ_c α_c ∫ f(p) / g(p) dr_c,   p = φ_c(G_c^{-1}(r_c)),        (Eq. 28)
 *     g(p) = Σ_c α_c g_c(x_c) / φ'_c(x_c),   x_c = φ_c^{-1}(p).        (Eq. 30)
 *
 * and turns the adapted grids into unweighted events by rejection against the
 * maximum weight (§2, Eq. 2; §3.5, last paragraph).
 *
 * Conventions shared by every entry point:
 *   - Every function returns a vamp_status; none aborts, traps or exits.
 *     vamp_last_error() gives a message for the last failure on a context.
 *   - All GPU work is enqueued on the CUDA stream given to vamp_create (NULL
 *     = the legacy default stream).  Entry points that hand results back in
 *     host memory synchronise that stream before returning.
 *   - A context owns every device buffer it uses (grids, α, accumulators,
 *     generation staging); inputs are copied at create time.  Event records
 *     are written into caller-owned device memory.
 *   - Arrays are row-major.  Grid edges are [K][d][n+1] (ξ_{c,k,j}), bin
 *     d-values [K][d][n], per-channel arrays [K].
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     (seed low word, seed high word); counter (call, word block, stream
 *     field, request id); word w of a call is lane w%4 of block w/4.
 *     Integration pass `iteration` uses stream field = iteration (< 2^31);
 *     generation batch b of call gen_id uses 0x80000000 | gen_id<<16 | b.
 *     A pass is therefore reproducible and independent of launch shape (§4.4).
 *   - Limits: 1 <= d <= 16, 1 <= n_bins <= 256, 1 <= K, at most 4 mapped
 *     coordinates per channel or peak, at most 2^32-1 calls per pass.
 */
#ifndef VAMP_H
#define VAMP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VAMP_OK = 0,
    VAMP_ERR_INVALID_ARG = 1, /* bad pointer, size or descriptor */
    VAMP_ERR_OOM = 2,         /* device or host allocation failed */
    VAMP_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the name) */
    VAMP_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    VAMP_ERR_NUMERIC = 5,     /* a non-finite weight was seen (the call still completed) */
    VAMP_ERR_STATE = 6,       /* call out of order, e.g. refine before any pass */
    VAMP_ERR_LIMIT = 7        /* a served request reached its generation call limit (events are partial) */
} vamp_status;

typedef enum {
    VAMP_PREC_FP64 = 0,      /* maps, integrand and g(p) in FP64 */
    VAMP_PREC_FP32_EVAL = 1  /* maps, integrand and g(p) in FP32; sums, grids, α in FP64 */
} vamp_precision;

typedef enum { VAMP_MAP_ID = 0, VAMP_MAP_BW = 1, VAMP_MAP_POW = 2 } vamp_map_kind;

typedef enum { VAMP_GAUSS_NORM_REAL_LINE = 0, VAMP_GAUSS_NORM_UNIT = 1 } vamp_gauss_norm;

/* Per-axis kind of a channel equivalence (§3.5): how the bin weights of the
 * matched axis of the partner channel enter the rebinning of this axis. */
typedef enum {
    VAMP_EQ_IDENTITY = 0,   /* bin j adds the partner's bin j */
    VAMP_EQ_INVERT = 1,     /* bin j adds the partner's bin n-1-j (mirrored axis) */
    VAMP_EQ_SYMMETRIC = 2,  /* bin j adds the mean of the partner's bins j and n-1-j */
    VAMP_EQ_INVARIANT = 3   /* the axis takes unit weights: rebinning keeps it */
} vamp_equiv_kind;

/* One channel map φ_c, or one integrand peak (same shape).  Slot s <
 * n_mapped maps coordinate coord[s]; all other coordinates are identity.
 *   VAMP_MAP_BW : Breit-Wigner, a = mass m, b = width Γ > 0;
 *                 p = m + Γ tan(A x - atan(m/Γ)), A = atan((1-m)/Γ) + atan(m/Γ),
 *                 density 1/φ' = Γ / (A ((p-m)^2 + Γ^2)).
 *   VAMP_MAP_POW: power law; as a channel map p = x^5 (density 0.2 p^-0.8);
 *                 as an integrand factor (p+δ)^-0.8 / (5((1+δ)^0.2 - δ^0.2)),
 *                 b = δ >= 0.
 * Coordinates within one descriptor are distinct. */
typedef struct {
    int32_t n_mapped;
    int32_t coord[4];
    int32_t kind[4];
    double a[4];
    double b[4];
} vamp_map_desc;

/* Problem and adaptation settings (all pointers are host memory, read during
 * vamp_create only).
 * Integrand (synthetic stand-in for the matrix element, §3.1):
 *   f(p) = Σ_q peak_weight[q] Π_k ( k mapped by peak q ? factor_q(p_k) : G(p_k) )
 *   G = Gaussian(gauss_centre, gauss_sigma) normalised on the real line or on
 *   [0,1] (gauss_norm); gauss_sigma = 0 makes G = 1.  Peak weights may be
 *   negative: f then takes both signs (§3.1), weights w = f/g are signed. */
typedef struct {
    int32_t d;                  /* dimensions, 1..16 */
    int32_t n_channels;         /* K >= 1 */
    int32_t n_bins;             /* bins per axis n, 1..256 */
    const vamp_map_desc *channels; /* [K] */
    int32_t n_peaks;            /* >= 1 */
    const double *peak_weight;  /* [n_peaks] */
    const vamp_map_desc *peaks; /* [n_peaks] */
    double gauss_sigma;
    double gauss_centre;
    int32_t gauss_norm;         /* vamp_gauss_norm */
    uint64_t seed;              /* Philox key */
    uint32_t request_id;        /* Philox counter word 3 */
    double grid_alpha;          /* power α of the rebinning measure (Eq. 14), e.g. 1.5 */
    double beta;                /* power β of the channel-weight update (Eq. 25), e.g. 0.5 */
    int64_t n_min;              /* lower threshold of calls per live channel, e.g. 10 (1..2^32-1) */
    int32_t smooth;             /* 1: 3-point average of the bin d-values before Eq. 14 */
    int32_t omega_mode;         /* ω_c of Eq. 25: 0 = channel variance V_c, 1 = second moment */
    int64_t gen_batch;          /* calls per generation batch (0 = 2^20), <= 2^24 */
    int32_t combine_from;       /* passes with iteration >= this enter the combination */
    int32_t precision;          /* vamp_precision */
    int32_t stratified;         /* 1: integration passes sample pseudo-stratified in r space (§3.3):
                                   per channel n_r = the largest m (<= 2^20) with 2 m^d <= N_c cells
                                   per axis, s = floor(N_c / n_r^d) calls per cell, N_c = s n_r^d;
                                   the per-call variance is the mean of the cells' sample variances.
                                   Generation stays importance sampling.  Contexts, batches and the
                                   request server (the allocation-free pass rejects it). */
    int32_t n_equiv;            /* channel equivalences (§3.5), 0..65536; 0 = none */
    const int32_t *equiv;       /* [n_equiv][2 + 2d] host, copied at creation: records
                                   (c, c', π_0..π_{d-1}, kind_0..kind_{d-1}).  Before each
                                   rebinning, axis k of channel c takes its own d-values plus, per
                                   record naming c (in table order), axis π_k of channel c' with
                                   kind_k (vamp_equiv_kind); all records read the pass's own
                                   d-values.  π must be a permutation of 0..d-1, c' may equal c.
                                   Contexts, batches and servers; the allocation-free pass, which
                                   does not rebin, accepts and ignores them. */
} vamp_config;

/* Result of one sampling pass (§3.1 Eqs. 10-11 per channel, Eq. 23 overall).
 *   integral  = Σ_c α_c I_c, I_c = mean weight of channel c's calls
 *   variance  = Σ_c α_c^2 V_c / N_c (squared error of `integral`)
 *   w_max     = largest |w| of the pass, efficiency = integral / w_max (Eq. 2; for
 *               integrands of both signs the net yield after cancellation) 
 *   combined, combined_sigma, chi2_dof: inverse-variance combination of the
 *   passes with iteration >= combine_from (0 while there are none). */
typedef struct {
    double integral;
    double variance;
    double w_max;
    double efficiency;
    int64_t n_calls;
    double combined;
    double combined_sigma;
    double chi2_dof;
} vamp_pass_result;

typedef struct vamp_ctx vamp_ctx;

/* Creates a context on the current CUDA device: uniform grids ξ_j = j/n and
 * α_c = 1/K (§3.4, §3.5).  Copies the descriptors; allocates device state.
 * cuda_stream: a cudaStream_t (may be NULL).  Errors: INVALID_ARG (bad
 * descriptor), OOM, CUDA.  *out is NULL on failure. */
vamp_status vamp_create(const vamp_config *cfg, void *cuda_stream, vamp_ctx **out);

/* One sampling pass with the current grids and α (§3.5 work order; by
 * importance, or pseudo-stratified in r space when cfg->stratified is set,
 * §3.3): N_c = max(n_min, floor(α_c n_calls)) calls per live channel (whole
 * cells of that size when stratified); each
 * call maps r -> x_c -> p, evaluates f, inverts every other channel for g(p),
 * and accumulates w = f/g into per-channel sums, the bin d-values
 * D_{c,k,j} = Σ w^2 (Eq. 15) and the maximum weight.  `iteration` (< 2^31)
 * selects the random stream.  `out` (host) is required; the call
 * synchronises the stream.  NUMERIC if a weight was not finite. */
vamp_status vamp_sample_pass(vamp_ctx *ctx, int64_t n_calls, uint32_t iteration,
                             vamp_pass_result *out);

/* Asynchronous form of vamp_sample_pass: enqueues the same pass on the
 * context's stream and returns without waiting.  When the stream reaches it,
 * dev_out (caller-owned device memory, 8-byte aligned, 9 doubles) receives
 * integral, variance, w_max, efficiency, n_calls, combined, combined_sigma,
 * chi2_dof (as in vamp_pass_result) and the device error flags (0: none;
 * non-zero: a non-finite weight or a wait that gave up, which the next
 * vamp_sample_pass or vamp_generate also reports and clears).  A context's
 * first pass picks its kernel by timing the candidates and synchronises;
 * once a pass of at least as many calls has run, the call allocates nothing
 * and only launches kernels and memsets, so an adaptation iteration
 * (this call, vamp_refine_grids, vamp_update_alpha) can be captured in a CUDA
 * graph.  Errors: INVALID_ARG as vamp_sample_pass, or for dev_out. */
vamp_status vamp_sample_pass_async(vamp_ctx *ctx, int64_t n_calls, uint32_t iteration, double *dev_out);

/* Rebins every (channel, axis) grid from the last pass's d-values (Eqs. 14,
 * 15): ω_j = sqrt(D_j), r_j = ω_j / Σ ω, m_j = ((r_j - 1)/ln r_j)^grid_alpha;
 * new edges invert the cumulative of m, linear inside each old bin.
 * Asynchronous.  STATE if no pass has run. */
vamp_status vamp_refine_grids(vamp_ctx *ctx);

/* Channel-weight update α_c <- α_c ω_c^β / Σ α ω^β (Eq. 25) from the last
 * pass.  Channels without variance keep α_c; channels whose calls all gave
 * w = 0 are switched off.  Asynchronous.  STATE if no pass has run. */
vamp_status vamp_update_alpha(vamp_ctx *ctx);

/* Unweighted events from the current grids and α (§3.5 last paragraph):
 * batches of gen_batch calls, channel drawn with probability α_c, accept
 * iff u w_max < |w|; the record keeps w with its sign, so integrands of both
 * signs (§3.1) give events of weight ±1 in units of w_max after the sign is
 * read.  w_max starts at the last pass's maximum |w| and is raised
 * to the batch maximum between batches.  The first n_events accepted events
 * in call order are written to dev_records (device memory, caller-owned,
 * n_events * vamp_record_bytes(d) bytes, 8-byte aligned): record i =
 * { float p[d]; zero padding to 8 bytes; double w }.  Outputs (host): events
 * written, calls consumed up to the last written event, overweight events
 * (|w| > w_max) among them.  Synchronises.  STATE if no pass has run;
 * TIMEOUT if 65536 batches did not yield n_events. */
vamp_status vamp_generate(vamp_ctx *ctx, int64_t n_events, uint32_t gen_id, void *dev_records,
                          int64_t *n_written, int64_t *n_calls_used, int64_t *n_overweight);

/* Bytes of one event record for dimension d: round_up(4 d, 8) + 8. */
int64_t vamp_record_bytes(int32_t d);

/* Copies the state to host arrays (any may be NULL): edges [K][d][n+1],
 * alpha [K], per-channel shifts [K] (previous pass means), w_max.
 * Synchronises.  Used for checkpoints and tests. */
vamp_status vamp_get_state(vamp_ctx *ctx, double *edges, double *alpha, double *shift,
                           double *w_max);

/* Overwrites the state from host arrays (NULL = keep).  Edges must be
 * strictly increasing from 0 to 1 on every row, α >= 0 with Σ α > 0.
 * Marks the context as having run a pass (so refine/generate are allowed).
 * Synchronises. */
/* Checkpoint of the adaptation state (the analogue of the grid file that
 * the paper's master writes after each iteration for restarts, §4.5): grids ξ,
 * α, channel shifts, generation w_max and the history of passes that the
 * iteration combination uses, as one self-describing host blob (magic
 * "VAMPCKP1", d, K, n, precision, then FP64 arrays).  vamp_checkpoint_bytes
 * gives the blob size (-1 on error; synchronises); vamp_checkpoint writes it
 * to host_buf (bytes >= that size); vamp_restore loads a blob of the same
 * (d, K, n) into a context (either precision: the master state is FP64),
 * validating it as vamp_set_state does.  A run restored after iteration i
 * continues as the uninterrupted run would (next pass: iteration i+1). */
int64_t vamp_checkpoint_bytes(vamp_ctx *ctx);
vamp_status vamp_checkpoint(vamp_ctx *ctx, void *host_buf, int64_t bytes);
vamp_status vamp_restore(vamp_ctx *ctx, const void *host_buf, int64_t bytes);

vamp_status vamp_set_state(vamp_ctx *ctx, const double *edges, const double *alpha,
                           const double *shift, double w_max);

/* Copies the last pass's per-channel data to host (any may be NULL): bin
 * d-values D [K][d][n], channel means I_c [K], variances V_c [K], calls
 * N_c [K].  Synchronises. */
vamp_status vamp_get_pass(vamp_ctx *ctx, double *D, double *Ic, double *Vc, int64_t *Nc);

/* Diagnostic: evaluates `count` single calls without accumulating, into host
 * arrays (any but fgwc may be NULL): x [count][d] channel coordinates,
 * p [count][d], jf [count][d] forward bins, bins [count][K][d] bin of every
 * channel's lookup (-1 for channels with α = 0), fgwc [count][4] =
 * {f, g, w, channel}.  mode 0: call `call0 + i` of the integration stream
 * `field` with the channel from the allocation of the last pass (or of
 * vamp_allocate); mode 1: generation call with the channel drawn from α.
 * Allocates temporary device memory; synchronises. */
vamp_status vamp_eval_calls(vamp_ctx *ctx, int32_t mode, uint32_t field, uint32_t call0,
                            int32_t count, double *x, double *p, int32_t *jf, int32_t *bins,
                            double *fgwc);

/* Computes the call allocation N_c for n_calls without sampling (used with
 * vamp_eval_calls).  Returns the total in *n_total.  Synchronises. */
vamp_status vamp_allocate(vamp_ctx *ctx, int64_t n_calls, int64_t *n_total);

/* Kernel timing for benchmarks: with enable = 1 the context records CUDA
 * events on its stream around every launch of the sampling kernel and of the
 * generation kernel; vamp_kernel_stats returns the summed device time (ms)
 * and the launch counts since the last enable (it synchronises the stream
 * when asynchronous passes are still pending; passes enqueued during a
 * stream capture are not timed).  Off by default. */
vamp_status vamp_profile(vamp_ctx *ctx, int32_t enable);

/* Self-test of the device-side bounded wait that every staged-tile wait of
 * the pass kernels uses: one CTA waits, with a limit of limit_cycles SM
 * cycles (1 .. 2^31), for an mbarrier phase that nothing completes.  Returns
 * VAMP_ERR_TIMEOUT when the wait gave up as designed (the device and every
 * context stay usable), VAMP_OK if it was not armed, INVALID_ARG / OOM /
 * CUDA otherwise; *waited_cycles (may be NULL) receives the cycles waited.
 * Synchronises the device's legacy default stream. */
vamp_status vamp_selftest_bounded_wait(int64_t limit_cycles, int64_t *waited_cycles);
vamp_status vamp_kernel_stats(vamp_ctx *ctx, double *sample_ms, int64_t *sample_launches, double *gen_ms,
                              int64_t *gen_launches);

/* The pass-kernel variant the context uses (chosen at create time by timing
 * the candidates once per process and shape class): FP32-eval or FP64, calls
 * per thread, the (d, n) it is specialised for (0, 0 = any shape) and the
 * CTAs per SM it is compiled for.  For benchmarks and profiles.  Any pointer
 * may be NULL. */
vamp_status vamp_pass_kernel_info(const vamp_ctx *ctx, int32_t *fp32, int32_t *calls_per_thread,
                                  int32_t *shape_d, int32_t *shape_n, int32_t *ctas_per_sm);

/* Throughput of this GPU's pipes, measured by small kernels that keep one
 * pipe busy (for the per-pipe roofline of the sampling kernel; the paper has
 * no counterpart).  Per second, summed over all SMs: FP32 fused
 * multiply-add lane-instructions (the issue rate of 32-bit arithmetic),
 * FP64 fused multiply-add lane-instructions, MUFU (special-function unit)
 * lane-instructions (2^x), shared-memory load wavefronts (one per warp
 * load of 32 consecutive words), and bytes read from L2 by coalesced
 * 16-byte loads that bypass L1 (a 32 MiB buffer resident in L2).  Runs on
 * the current device and synchronises it; takes a few tens of
 * milliseconds.  OOM / CUDA on failure. */
typedef struct vamp_pipe_peaks {
    double fp32_lane_ops;
    double fp64_lane_ops;
    double xu_lane_ops;
    double lds_wavefronts;
    double l2_read_bytes;
} vamp_pipe_peaks;
vamp_status vamp_measure_peaks(vamp_pipe_peaks *out);

/* Name of the pass kernel the context uses for mode 0 (integration) or 1
 * (generation), as profilers print it, e.g. "k_pass<float, 0, 2, 14, 100, 2>",
 * written NUL-terminated into buf (len bytes, host).  INVALID_ARG for a bad
 * mode or a buffer too small. */
vamp_status vamp_pass_kernel_name(const vamp_ctx *ctx, int32_t mode, char *buf, int32_t len);

/* Number of compiled pass-kernel variants that can run this context's shape
 * and sampling mode: the autotuner's candidates, in a fixed order
 * (shape-specialised staged-tile kernels "k_pass" first, then the generic
 * one; for FP32-eval importance sampling with K <= 64 and K (n+1) <= 16384,
 * then the union kernels "k_union", which find every channel's bin of p_k
 * with one search in per-coordinate tables of all channels' edge images,
 * Eq. 30 evaluated the same way). */
vamp_status vamp_pass_kernel_candidates(const vamp_ctx *ctx, int32_t *count);

/* Pins the context's pass kernels (integration and generation) to candidate
 * `index` (0 <= index < count of vamp_pass_kernel_candidates) instead of the
 * autotuner's pick at the first pass -- for tests that must run a given
 * variant and for reproducible timing.  Every candidate computes the same
 * pass; sums may differ in the order of floating-point additions (and, in
 * the FP32-eval form, in FP32 rounding).  The choice holds until the
 * context is destroyed.  While a union kernel is in use (picked here or by
 * the autotuner) the context also holds its interval tables on the device,
 * about d K (n+1) 264 + d 2^18 bytes (27.6 MB for d = 14, K = 64, n = 100),
 * rebuilt by every rebinning and state upload; choosing a staged-tile
 * kernel frees them.  INVALID_ARG for a bad index; OOM if the tables cannot
 * be allocated; CUDA if the kernel's shared memory cannot be configured.
 * (The autotuner itself, where the device has no room for the tables,
 * chooses among the staged-tile kernels alone and does not remember that
 * choice for later contexts.) */
vamp_status vamp_select_pass_kernel(vamp_ctx *ctx, int32_t index);

/* ---- many independent integrations in one launch --------------------------
 * A batch advances n integrations of possibly different d, K, n, calls and
 * seeds together (all in the same precision): every iteration runs ONE
 * persistent pass kernel whose CTAs take work items -- up to item_calls
 * consecutive calls of one channel of one instance -- from an atomic counter,
 * plus a few multi-instance kernels for allocation, pass results, rebinning
 * and α.  The paper's analogue is the automatic choice between parallel
 * modes over channels and over stratification cells (§4.5.2).  Each
 * iteration is captured once as a CUDA graph and replayed.  Results equal
 * those of running every instance alone with vamp_create /
 * vamp_sample_pass / vamp_refine_grids / vamp_update_alpha (same random
 * streams), up to the order of floating-point sums. */
typedef struct vamp_batch vamp_batch;

/* Creates the batch on the current device with its own CUDA stream; cfgs[i]
 * as for vamp_create (all with the same precision).  autotune_tiles = 1: the
 * first iteration times work-item sizes (512, 1024, 2048, 4096, 8192 calls) and
 * shared-memory budgets (112 KB per CTA with two CTAs per SM, or, in the
 * FP32-eval form, 72 KB with three) once and keeps the fastest; 0: 512 calls
 * per item, 112 KB per CTA. */
vamp_status vamp_batch_create(const vamp_config *cfgs, int32_t n, int32_t autotune_tiles, vamp_batch **out);

/* One adaptation iteration of every instance: n_calls[i] calls (host array),
 * random stream `iteration` (< 2^31), adapt bit 0 = rebin grids, bit 1 =
 * update α; results[i] (host array of n) receive the pass results.
 * Synchronises.  NUMERIC / TIMEOUT as for vamp_sample_pass. */
vamp_status vamp_batch_iterate(vamp_batch *b, const int64_t *n_calls, uint32_t iteration, int32_t adapt,
                               vamp_pass_result *results);

/* State of one instance into host arrays (any may be NULL), as vamp_get_state. */
vamp_status vamp_batch_get_state(vamp_batch *b, int32_t instance, double *edges, double *alpha, double *shift,
                                 double *w_max);

/* The launch shape in use and the autotuner's timings of one pass (tuned and
 * fixed shape, at the first iteration's calls; 0 if untuned). */
vamp_status vamp_batch_tuning(const vamp_batch *b, int64_t *item_calls, int32_t *budget_kb, double *tuned_ms,
                              double *fixed_ms);

void vamp_batch_destroy(vamp_batch *b);
const char *vamp_batch_last_error(const vamp_batch *b);

/* ---- request serving with continuous batching -----------------------------
 * A request is one whole use of the method (§3, §3.5): `iterations`
 * adaptation iterations of `calls` calls each (rebinning, Eq. 14, and α
 * update, Eq. 25, after every pass; passes from combine_from on are
 * combined), then n_events unweighted events (§3.5) from the adapted grids,
 * generation stream gen_id = 0.  A scheduler thread admits queued requests
 * while fewer than max_slots are active and their device memory stays within
 * mem_budget_bytes (a request that alone exceeds the budget runs when nothing
 * else does); every scheduler tick advances all integrating requests by one
 * iteration in one multi-instance launch (a request that arrives meanwhile
 * joins the next tick) and keeps one generation batch of every generating
 * request in flight on the request's own stream.  Each request's results and
 * events equal those of the same request run alone through vamp_create /
 * vamp_sample_pass (iteration i) / vamp_refine_grids / vamp_update_alpha /
 * vamp_generate(gen_id 0), up to the order of floating-point sums. */
typedef struct vamp_server vamp_server;

typedef struct vamp_request_result {
    uint64_t id;
    int32_t status;             /* vamp_status of the request */
    int32_t iterations;         /* iterations completed */
    vamp_pass_result result;    /* the last pass, with the running combination */
    int64_t calls_total;        /* Σ N' over the iterations */
    int64_t events_written;
    int64_t events_calls_used;
    int64_t events_overweight;
    double queue_s;             /* submit -> admission (seconds) */
    double latency_s;           /* submit -> completion (seconds) */
} vamp_request_result;

/* Starts the scheduler thread on the current device.  precision: every
 * request is run in this precision (its cfg->precision is ignored). */
vamp_status vamp_server_create(int32_t max_slots, int64_t mem_budget_bytes, int32_t precision, vamp_server **out);

/* Queues a request (cfg copied during the call).  iterations >= 1;
 * calls >= 1; max_gen_calls: generation stops after the first batch that
 * brings the calls spent on events to at least this many (0 = at most 2^16
 * batches) and the request ends with VAMP_ERR_LIMIT and the events so far --
 * a poorly adapted request can have a tiny unweighting efficiency; dev_records: device buffer of n_events *
 * vamp_record_bytes(cfg->d) bytes, 8-byte aligned, owned by the caller and
 * left untouched by anything but this request until its result is polled
 * (may be NULL when n_events = 0).  *id_out receives the request id.
 * INVALID_ARG for a bad cfg or arguments; nothing is queued then. */
vamp_status vamp_server_submit(vamp_server *s, const vamp_config *cfg, int32_t iterations, int64_t calls,
                               int64_t n_events, int64_t max_gen_calls, void *dev_records, uint64_t *id_out);

/* vamp_server_submit that also hands back the adapted state (the analogue of
 * the paper's grid files, §4.5): dev_state (device, 8-byte aligned, owned by
 * the caller and left untouched by anything but this request until its
 * result is polled; NULL = none) receives, once the last adaptation
 * iteration is done, the grids [K][d][n+1], α [K] and the channel shifts
 * [K] (FP64, K*d*(n+1) + 2K doubles) -- what vamp_get_state returns for the
 * same request run alone.  The copy is complete when the request's result
 * is polled. */
vamp_status vamp_server_submit_state(vamp_server *s, const vamp_config *cfg, int32_t iterations, int64_t calls,
                                     int64_t n_events, int64_t max_gen_calls, void *dev_records, double *dev_state,
                                     uint64_t *id_out);

/* Moves up to max_results completed requests (completion order) into out
 * (host); returns how many. */
int32_t vamp_server_poll(vamp_server *s, vamp_request_result *out, int32_t max_results);

/* Waits until no request is queued or active (TIMEOUT after timeout_s). */
vamp_status vamp_server_wait_idle(vamp_server *s, double timeout_s);

/* Counters since creation: scheduler ticks that ran an integration launch,
 * integration calls, events written; device bytes held by active requests. */
vamp_status vamp_server_stats(const vamp_server *s, int64_t *ticks, int64_t *calls, int64_t *events,
                              int64_t *mem_in_use);

/* Scheduler load as of its last tick: requests queued, integrating and
 * generating; generation batches launched since creation. */
vamp_status vamp_server_load(const vamp_server *s, int32_t *queued, int32_t *integrating, int32_t *generating,
                             int64_t *gen_batches);

/* Stops the scheduler (queued requests are dropped; active ones are left
 * unfinished) and frees everything. */
void vamp_server_destroy(vamp_server *s);

/* One sampling pass that makes no device-memory allocation, for callers that
 * cannot let a library allocate device memory (all of it owned by the
 * caller's own pool, or a path where an allocation could block or fail
 * unpredictably).  The paper has no counterpart: it is an interface addition
 * of this library.  (Host-side set-up uses small temporary heap buffers.)
 *
 * Same pass as vamp_sample_pass, without a context, run by the first
 * candidate kernel of the shape (vamp_pass_kernel_candidates order; a
 * context pinned to it gives the same sums): the caller passes the
 * problem (cfg, host memory, read during the call), the grid state in device
 * memory -- dev_edges [K][d][n+1], dev_alpha [K], dev_shift [K] (previous
 * pass means, zeros for a first pass), all read only -- and the outputs:
 * dev_D_out (device, [K][d][n] bin d-values of the pass, may be NULL) and
 * out (host).  The combination fields of *out are 0.  err_msg (optional,
 * err_len bytes) receives a message on failure.
 *
 * All working arrays live in one static device array of 8 MiB that every
 * GPU loading this library's device code holds until the process exits; a
 * problem that needs more (about K * d * (n+1) * 32 bytes plus small terms)
 * is rejected with VAMP_ERR_INVALID_ARG and a message.  Under CUDA's default
 * lazy module loading the array comes into being with the module at the
 * first call on a device (at module load otherwise): make that first call
 * before a pool of yours reserves all free device memory, and before any
 * stream capture.  The array's address is looked up on every call in the
 * current context, so it stays right after a device reset.  The call clears
 * what must start at zero; calls that overlap on the GPU share the array and
 * race.  Synchronises cuda_stream. */
vamp_status vamp_sample_pass_static(const vamp_config *cfg, const double *dev_edges, const double *dev_alpha,
                                    const double *dev_shift, int64_t n_calls, uint32_t iteration,
                                    void *cuda_stream, double *dev_D_out, vamp_pass_result *out,
                                    char *err_msg, int32_t err_len);

/* Releases all device and host memory of the context (NULL is allowed). */
void vamp_destroy(vamp_ctx *ctx);

/* Message of the last failure on ctx (never NULL; empty when none). */
const char *vamp_last_error(const vamp_ctx *ctx);

/* Static name of a status code. */
const char *vamp_status_string(vamp_status s);

/* SHA-256 (hex) of the sources, headers and compiler flags this library was
 * built from (static string; "unknown" for a build outside the in-tree build
 * script).  Lets a caller check that the binary is the one its sources
 * describe. */
const char *vamp_source_hash(void);

#ifdef __cplusplus
}
#endif
#endif /* VAMP_H */

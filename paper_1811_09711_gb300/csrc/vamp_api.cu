// vamp_api.cu -- the C ABI of include/vamp.h: contexts, launch order,
// result read-back, and the choice of pass-kernel variant (autotuned once per
// shape class).  Every step of the integration runs in the kernels; this file
// only marshals.
#include "../../include/vamp.h"
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

using vamp::Params;
using vamp::PassVariant;
using vamp::Scalars;

struct vamp_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int d = 0, K = 0, n = 0, P = 0;
    int fp32 = 0;
    int combine_from = 0;
    int64_t gen_batch = 1 << 20;
    int sm_count = 0;
    int tile = 1;              // channels per staged tile
    size_t smem_pass = 0;      // dynamic shared memory of the integration pass kernel
    size_t smem_gen = 0;       // ... of the generation pass kernel
    const PassVariant* var = nullptr;  // pass kernels in use
    void* uni_buf = nullptr;   // interval tables of the union pass (allocated while such a kernel is in use)
    int uni_on = 0;            // the tables exist and follow every grid change
    int tuned = 0;             // var was chosen by timing (first sampling pass)
    int64_t cell_cap = 0;      // cells the stratified-pass cell sums hold
    int grid_pass = 0;         // persistent grid of the integration pass kernel
    int grid_gen = 0;          // resident CTAs of the generation pass kernel
    int have_pass = 0;
    Params prm{};
    void* arena = nullptr;
    Scalars* h_head = nullptr;   // pinned copy of the Scalars head
    // generation staging (allocated on first use)
    unsigned char* g_staging = nullptr;
    uint32_t* g_callidx = nullptr;
    int* g_counts = nullptr;
    long long* g_offsets = nullptr;
    int64_t g_cap = 0;            // calls (slots) the staging holds
    // kernel timing (vamp_profile)
    int prof = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    double prof_sample_ms = 0.0, prof_gen_ms = 0.0;
    int64_t prof_sample_n = 0, prof_gen_n = 0;
    // event pairs around asynchronous passes, read by vamp_kernel_stats
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    std::string err;
};

namespace {

constexpr size_t HEAD_BYTES = offsetof(Scalars, n_hist) + sizeof(int32_t) * 2;

vamp_status fail(vamp_ctx* c, vamp_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

vamp_status cuda_fail(vamp_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, VAMP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define VAMP_CK(ctx, call)                                             \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
    } while (0)

// Keeps the context's device current for the duration of an entry point.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

vamp_status read_head(vamp_ctx* c)
{
    VAMP_CK(c, cudaMemcpyAsync(c->h_head, c->prm.sc, HEAD_BYTES, cudaMemcpyDeviceToHost, c->stream));
    VAMP_CK(c, cudaStreamSynchronize(c->stream));
    return VAMP_OK;
}

vamp_status take_numeric_flag(vamp_ctx* c)
{
    const unsigned err = c->h_head->err;
    if (err) {
        const unsigned zero = 0;
        VAMP_CK(c, cudaMemcpyAsync(&c->prm.sc->err, &zero, sizeof zero, cudaMemcpyHostToDevice, c->stream));
        VAMP_CK(c, cudaStreamSynchronize(c->stream));
        if (err & vamp::ERR_TIMEOUT)
            return fail(c, VAMP_ERR_TIMEOUT, "a bounded wait for staged grid data gave up; results are incomplete");
        return fail(c, VAMP_ERR_NUMERIC, "a non-finite weight was produced (counted as w = 0)");
    }
    return VAMP_OK;
}

vamp::PassArgs pass_args(const vamp_ctx* c, uint32_t field)
{
    vamp::PassArgs A{};
    A.field = field;
    A.tile = c->tile;
    A.ntiles = (c->K + c->tile - 1) / c->tile;
    return A;
}

// Autotuner: the fastest pass-kernel variant for a shape class and call
// count (power-of-two class), measured once per process on a pass of the
// context's first call count and then reused.
std::mutex g_tune_mu;
// key: device, precision, d, n, K (capped), call-count class, pseudo-stratified (whose candidates
// are the generic kernels only)
std::map<std::tuple<int, int, int, int, int, int, int>, const PassVariant*> g_tuned;

// Tile and shared memory of one candidate (its CTAs-per-SM budget).
struct VariantShape {
    int tile;
    size_t smem_pass, smem_gen;
};

VariantShape shape_of(const vamp_ctx* c, const PassVariant* v)
{
    VariantShape s{};
    if (v->uni) {
        s.tile = 1;
        s.smem_pass = vamp::union_pass_smem(c->prm, *v, 0);
        s.smem_gen = vamp::union_pass_smem(c->prm, *v, 1);
        return s;
    }
    vamp::pass_smem_for(c->prm, c->fp32, v->minb, &s.tile, &s.smem_pass, &s.smem_gen);
    return s;
}

// Allocates the union pass's interval tables once; false (and the
// allocation error cleared) where the device has no room for them.
bool union_alloc(vamp_ctx* c)
{
    if (c->uni_buf) return true;
    void* b = nullptr;
    if (cudaMalloc(&b, vamp::union_bytes(c->d, c->K, c->n)) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    c->uni_buf = b;
    vamp::bind_union(c->prm, (unsigned char*)b);
    return true;
}

// Allocates the interval tables and enqueues their build from the current
// grids; from then on every grid change rebuilds them.
vamp_status union_enable(vamp_ctx* c)
{
    if (!union_alloc(c)) return fail(c, VAMP_ERR_OOM, "interval tables of the union pass");
    VAMP_CK(c, vamp::launch_union_build(c->prm, c->stream));
    c->uni_on = 1;
    return VAMP_OK;
}

void union_disable(vamp_ctx* c)
{
    if (c->uni_buf) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->uni_buf);
    }
    c->uni_buf = nullptr;
    c->uni_on = 0;
    vamp::bind_union(c->prm, nullptr);
}

std::vector<const PassVariant*> candidates_of(const vamp_ctx* c)
{
    return vamp::pass_candidates(c->fp32, c->d, c->n, c->prm.stratified, c->K);
}

// Makes v the context's pass kernel: its tile, shared memory and grids.
vamp_status use_variant(vamp_ctx* c, const PassVariant* v)
{
    if (v->uni && !c->uni_on) {
        const vamp_status us = union_enable(c);
        if (us != VAMP_OK) return us;
    } else if (!v->uni && c->uni_buf) {
        union_disable(c);
    }
    const VariantShape s = shape_of(c, v);
    VAMP_CK(c, vamp::ensure_smem(v->fn[0], s.smem_pass));
    VAMP_CK(c, vamp::ensure_smem(v->fn[1], s.smem_gen));
    int b0 = 0, b1 = 0;
    VAMP_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, v->fn[0], vamp::PASS_THREADS, s.smem_pass));
    VAMP_CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, v->fn[1], vamp::PASS_THREADS, s.smem_gen));
    c->var = v;
    c->tile = s.tile;
    c->smem_pass = s.smem_pass;
    c->smem_gen = s.smem_gen;
    c->grid_pass = (b0 > 0 ? b0 : 1) * c->sm_count;
    c->grid_gen = (b1 > 0 ? b1 : 1) * c->sm_count;
    return VAMP_OK;
}

vamp_status choose_variant(vamp_ctx* c, int64_t n_calls)
{
    std::vector<const PassVariant*> cand = candidates_of(c);
    // the union kernels run on their interval tables: where the device has
    // no room for those, the staged-tile kernels are chosen among alone
    const bool any_uni = std::any_of(cand.begin(), cand.end(), [](const PassVariant* v) { return v->uni != 0; });
    const bool reduced = any_uni && !union_alloc(c);
    if (reduced)
        cand.erase(std::remove_if(cand.begin(), cand.end(), [](const PassVariant* v) { return v->uni != 0; }),
                   cand.end());
    if (cand.empty()) return fail(c, VAMP_ERR_INVALID_ARG, "no pass kernel for this shape");
    for (const PassVariant* v : cand) {
        const VariantShape s = shape_of(c, v);
        VAMP_CK(c, vamp::ensure_smem(v->fn[0], s.smem_pass));
        VAMP_CK(c, vamp::ensure_smem(v->fn[1], s.smem_gen));
    }
    auto grid_of = [&](const PassVariant* v, int mode, int* grid) -> cudaError_t {
        const VariantShape s = shape_of(c, v);
        int b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, v->fn[mode], vamp::PASS_THREADS,
                                                                      mode ? s.smem_gen : s.smem_pass);
        *grid = (b > 0 ? b : 1) * c->sm_count;
        return e;
    };
    const int64_t probe = std::min<int64_t>(std::max<int64_t>(n_calls, 1 << 16), 1 << 24);
    int nclass = 0;
    while ((int64_t(1) << (nclass + 1)) <= probe) ++nclass;
    const auto key = std::make_tuple(c->dev, c->fp32, c->d, c->n, std::min(c->K, 64), nclass, c->prm.stratified);
    const PassVariant* best = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) best = it->second;
    }
    if (best && std::find(cand.begin(), cand.end(), best) == cand.end()) best = nullptr;  // not a candidate here
    if (!best && cand.size() == 1) best = cand[0];
    if (!best) {
        // time each candidate on a pass of `probe` calls over the current
        // grids; the pass result is discarded (no finish kernel runs) and
        // the accumulators are cleared again below
        for (const PassVariant* v : cand)
            if (v->uni && !c->uni_on) {
                const vamp_status us = union_enable(c);
                if (us != VAMP_OK) return us;
            }
        cudaEvent_t e0, e1;
        VAMP_CK(c, cudaEventCreate(&e0));
        VAMP_CK(c, cudaEventCreate(&e1));
        float best_ms = 1e30f;
        for (const PassVariant* v : cand) {
            int grid = 0;
            VAMP_CK(c, grid_of(v, 0, &grid));
            const VariantShape s = shape_of(c, v);
            vamp::PassArgs A = pass_args(c, 0x7fffffffu);
            A.tile = s.tile;
            A.ntiles = (c->K + s.tile - 1) / s.tile;
            float ms_v = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                VAMP_CK(c, vamp::launch_begin_pass(c->prm, probe, c->stream));
                VAMP_CK(c, cudaEventRecord(e0, c->stream));
                VAMP_CK(c, v->launch(c->prm, 0, A, grid, s.smem_pass, c->stream));
                VAMP_CK(c, cudaEventRecord(e1, c->stream));
                VAMP_CK(c, cudaEventSynchronize(e1));
                VAMP_CK(c, cudaEventElapsedTime(&ms_v, e0, e1));
            }
            if (ms_v < best_ms) { best_ms = ms_v; best = v; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        // the probe touched the accumulators and the pass scalars (not the
        // combination history: tuning runs before the first pass)
        VAMP_CK(c, cudaMemsetAsync(c->prm.D, 0, (size_t)c->K * c->d * c->n * 8, c->stream));
        VAMP_CK(c, cudaMemsetAsync(c->prm.csum, 0, (size_t)2 * c->K * 8, c->stream));
        VAMP_CK(c, cudaMemsetAsync(c->prm.sc, 0, HEAD_BYTES, c->stream));
        VAMP_CK(c, cudaStreamSynchronize(c->stream));
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (!reduced) g_tuned[key] = best;  // a choice made without the union kernels is not kept
    }
    return use_variant(c, best);
}

}  // namespace

extern "C" {

const char* vamp_status_string(vamp_status s)
{
    switch (s) {
    case VAMP_OK: return "VAMP_OK";
    case VAMP_ERR_INVALID_ARG: return "VAMP_ERR_INVALID_ARG";
    case VAMP_ERR_OOM: return "VAMP_ERR_OOM";
    case VAMP_ERR_CUDA: return "VAMP_ERR_CUDA";
    case VAMP_ERR_TIMEOUT: return "VAMP_ERR_TIMEOUT";
    case VAMP_ERR_NUMERIC: return "VAMP_ERR_NUMERIC";
    case VAMP_ERR_STATE: return "VAMP_ERR_STATE";
    case VAMP_ERR_LIMIT: return "VAMP_ERR_LIMIT";
    }
    return "VAMP_ERR_UNKNOWN";
}

const char* vamp_last_error(const vamp_ctx* c) { return c ? c->err.c_str() : ""; }

#ifndef VAMP_SOURCE_HASH
#define VAMP_SOURCE_HASH "unknown"
#endif
const char* vamp_source_hash(void) { return VAMP_SOURCE_HASH; }

int64_t vamp_record_bytes(int32_t d) { return ((4 * (int64_t)d + 7) & ~int64_t(7)) + 8; }

void vamp_destroy(vamp_ctx* c)
{
    if (!c) return;
    {
        DeviceGuard g(c->dev);
        if (c->stream) cudaStreamSynchronize(c->stream);
        cudaFree(c->arena);
        cudaFree(c->uni_buf);
        cudaFree(c->prm.cellsum);
        cudaFree(c->g_staging);
        cudaFree(c->g_callidx);
        cudaFree(c->g_counts);
        cudaFree(c->g_offsets);
        cudaFreeHost(c->h_head);
        if (c->ev[0]) cudaEventDestroy(c->ev[0]);
        if (c->ev[1]) cudaEventDestroy(c->ev[1]);
        for (auto& pr : c->prof_pending) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
        for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    }
    delete c;
}

vamp_status vamp_create(const vamp_config* cfg, void* cuda_stream, vamp_ctx** out)
{
    if (!out) return VAMP_ERR_INVALID_ARG;
    *out = nullptr;
    Params pr{};
    vamp::Setup S;
    std::string why;
    if (!vamp::build_setup(cfg, pr, S, why)) return VAMP_ERR_INVALID_ARG;

    vamp_ctx* c = new (std::nothrow) vamp_ctx();
    if (!c) return VAMP_ERR_OOM;
    if (cudaGetDevice(&c->dev) != cudaSuccess) { delete c; return VAMP_ERR_CUDA; }
    c->stream = (cudaStream_t)cuda_stream;
    c->d = S.d; c->K = S.K; c->n = S.n; c->P = S.P;
    c->fp32 = S.fp32;
    c->combine_from = cfg->combine_from;
    c->gen_batch = cfg->gen_batch > 0 ? cfg->gen_batch : (int64_t(1) << 20);
    const vamp::Arena ar = vamp::plan_arena(pr);
    DeviceGuard g(c->dev);
    cudaError_t e = cudaMalloc(&c->arena, ar.bytes);
    if (e != cudaSuccess) { delete c; return e == cudaErrorMemoryAllocation ? VAMP_ERR_OOM : VAMP_ERR_CUDA; }
    e = cudaMallocHost((void**)&c->h_head, sizeof(Scalars));
    if (e != cudaSuccess) { vamp_destroy(c); return VAMP_ERR_OOM; }
    vamp::bind_arena(pr, (unsigned char*)c->arena, ar);
    c->prm = pr;
    Params& P = c->prm;

    // initial state: uniform grids ξ_j = j/n, α_c = 1/K (§3.4, §3.5)
    const int d = S.d, K = S.K, n = S.n;
    const size_t rows = (size_t)K * d;
    std::vector<double> edges(rows * (n + 1)), alpha(K, 1.0 / (double)K);
    for (size_t r = 0; r < rows; ++r)
        for (int j = 0; j <= n; ++j) edges[r * (n + 1) + j] = (double)j / (double)n;
    vamp_status st = VAMP_OK;
#define CREATE_CK(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) { st = cuda_fail(c, e_, #call); goto create_fail; }        \
    } while (0)
    CREATE_CK(cudaMemsetAsync(c->arena, 0, ar.bytes, c->stream));
    CREATE_CK(cudaMemcpyAsync(P.edges64, edges.data(), edges.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(cudaMemcpyAsync(P.alpha, alpha.data(), K * 8, cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(vamp::upload_setup(P, S, c->stream));
    CREATE_CK(vamp::launch_derive(P, c->stream));
    CREATE_CK(cudaStreamSynchronize(c->stream));
    {
        vamp::pass_smem(P, c->fp32, &c->tile, &c->smem_pass, &c->smem_gen);
        int maxsm = 0;
        CREATE_CK(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
        if ((int)c->smem_pass > maxsm) { st = fail(c, VAMP_ERR_INVALID_ARG, "grid too large for shared memory"); goto create_fail; }
        CREATE_CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev));
        // until the first pass picks by timing: the first candidate (the
        // shape-specialised kernel if there is one)
        const std::vector<const PassVariant*> cand = candidates_of(c);
        if (cand.empty()) { st = fail(c, VAMP_ERR_INVALID_ARG, "no pass kernel for this shape"); goto create_fail; }
        st = use_variant(c, cand[0]);
        if (st != VAMP_OK) goto create_fail;
    }
#undef CREATE_CK
    *out = c;
    return VAMP_OK;
create_fail:
    vamp_destroy(c);
    return st;
}

vamp_status vamp_allocate(vamp_ctx* c, int64_t n_calls, int64_t* n_total)
{
    if (!c || n_calls < 1) return fail(c, VAMP_ERR_INVALID_ARG, "n_calls must be >= 1");
    if (n_calls > int64_t(0xffffffff) || n_calls > int64_t(0xffffffff) - (int64_t)c->K * c->prm.n_min)
        return fail(c, VAMP_ERR_INVALID_ARG, "too many calls for a 32-bit call counter");
    DeviceGuard g(c->dev);
    VAMP_CK(c, vamp::launch_begin_pass(c->prm, n_calls, c->stream));
    vamp_status s = read_head(c);
    if (s != VAMP_OK) return s;
    if (n_total) *n_total = c->h_head->n_total;
    return VAMP_OK;
}

namespace {

// Checks, buffer sizing, kernel choice and the launches of one sampling pass
// (allocation, pass, stratified cell sums, result); nothing waits for them.
vamp_status enqueue_pass(vamp_ctx* c, int64_t n_calls, uint32_t iteration, cudaEvent_t e0, cudaEvent_t e1)
{
    if (n_calls < 1) return fail(c, VAMP_ERR_INVALID_ARG, "n_calls must be >= 1");
    if (iteration >= 0x80000000u) return fail(c, VAMP_ERR_INVALID_ARG, "iteration must be < 2^31");
    if (n_calls > int64_t(0xffffffff) || n_calls > int64_t(0xffffffff) - (int64_t)c->K * c->prm.n_min)
        return fail(c, VAMP_ERR_INVALID_ARG, "too many calls for a 32-bit call counter");
    DeviceGuard g(c->dev);
    // stratified passes: cell sums for at most (N + K n_min) / 2 cells (two
    // calls or more per cell), grown on demand
    const int64_t max_cells = c->prm.stratified ? (n_calls + (int64_t)c->K * c->prm.n_min) / 2 + c->K : 0;
    if (max_cells > c->cell_cap) {
        cudaFree(c->prm.cellsum);
        c->prm.cellsum = nullptr;
        c->cell_cap = 0;
        if (cudaMalloc(&c->prm.cellsum, (size_t)max_cells * 8) != cudaSuccess) {
            c->prm.cellsum = nullptr;
            return fail(c, VAMP_ERR_OOM, "cell sums of a stratified pass");
        }
        c->cell_cap = max_cells;
    }
    if (!c->tuned) {
        const vamp_status ts = choose_variant(c, n_calls);
        if (ts != VAMP_OK) return ts;
        c->tuned = 1;
    }
    const Params& P = c->prm;
    VAMP_CK(c, cudaMemsetAsync(P.D, 0, (size_t)c->K * c->d * c->n * 8, c->stream));
    VAMP_CK(c, cudaMemsetAsync(P.csum, 0, (size_t)2 * c->K * 8, c->stream));
    if (P.stratified) VAMP_CK(c, cudaMemsetAsync(P.cellsum, 0, (size_t)max_cells * 8, c->stream));
    VAMP_CK(c, vamp::launch_begin_pass(P, n_calls, c->stream));
    if (e0) VAMP_CK(c, cudaEventRecord(e0, c->stream));
    VAMP_CK(c, c->var->launch(P, 0, pass_args(c, iteration), c->grid_pass, c->smem_pass, c->stream));
    if (e1) VAMP_CK(c, cudaEventRecord(e1, c->stream));
    if (P.stratified) VAMP_CK(c, vamp::launch_strat_q(P, c->stream));
    VAMP_CK(c, vamp::launch_finish_pass(P, (int)iteration >= c->combine_from ? 1 : 0, c->stream));
    return VAMP_OK;
}

}  // namespace

vamp_status vamp_sample_pass(vamp_ctx* c, int64_t n_calls, uint32_t iteration, vamp_pass_result* out)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!out) return fail(c, VAMP_ERR_INVALID_ARG, "out is required");
    DeviceGuard g(c->dev);
    vamp_status s = enqueue_pass(c, n_calls, iteration, c->prof ? c->ev[0] : nullptr, c->prof ? c->ev[1] : nullptr);
    if (s != VAMP_OK) return s;
    s = read_head(c);
    if (s != VAMP_OK) return s;
    if (c->prof) {
        float ms = 0.f;
        VAMP_CK(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->prof_sample_ms += ms;
        c->prof_sample_n += 1;
    }
    const Scalars* h = c->h_head;
    out->integral = h->res[0];
    out->variance = h->res[1];
    out->w_max = h->res[2];
    out->efficiency = h->res[3];
    out->n_calls = h->n_total;
    out->combined = h->res[5];
    out->combined_sigma = h->res[6];
    out->chi2_dof = h->res[7];
    c->have_pass = 1;
    return take_numeric_flag(c);
}

vamp_status vamp_sample_pass_async(vamp_ctx* c, int64_t n_calls, uint32_t iteration, double* dev_out)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!dev_out || ((uintptr_t)dev_out & 7u)) return fail(c, VAMP_ERR_INVALID_ARG, "dev_out must be 8-byte aligned device memory");
    DeviceGuard g(c->dev);
    // kernel timing (vamp_profile) only outside a stream capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    VAMP_CK(c, cudaStreamIsCapturing(c->stream, &cap));
    cudaEvent_t e[2] = {nullptr, nullptr};
    if (c->prof && cap == cudaStreamCaptureStatusNone) {
        for (int q = 0; q < 2; ++q) {
            if (!c->ev_pool.empty()) { e[q] = c->ev_pool.back(); c->ev_pool.pop_back(); }
            else VAMP_CK(c, cudaEventCreate(&e[q]));
        }
        c->prof_pending.emplace_back(e[0], e[1]);
    }
    vamp_status s = enqueue_pass(c, n_calls, iteration, e[0], e[1]);
    if (s != VAMP_OK) return s;
    VAMP_CK(c, vamp::launch_pass_result(c->prm, dev_out, c->stream));
    c->have_pass = 1;
    return VAMP_OK;
}

vamp_status vamp_refine_grids(vamp_ctx* c)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!c->have_pass) return fail(c, VAMP_ERR_STATE, "refine before any sampling pass");
    DeviceGuard g(c->dev);
    VAMP_CK(c, vamp::launch_refine(c->prm, c->stream));
    if (c->uni_on) VAMP_CK(c, vamp::launch_union_build(c->prm, c->stream));
    return VAMP_OK;
}

vamp_status vamp_update_alpha(vamp_ctx* c)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!c->have_pass) return fail(c, VAMP_ERR_STATE, "alpha update before any sampling pass");
    DeviceGuard g(c->dev);
    VAMP_CK(c, vamp::launch_update_alpha(c->prm, c->stream));
    return VAMP_OK;
}

vamp_status vamp_generate(vamp_ctx* c, int64_t n_events, uint32_t gen_id, void* dev_records, int64_t* n_written,
                          int64_t* n_calls_used, int64_t* n_overweight)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!c->have_pass) return fail(c, VAMP_ERR_STATE, "generate before any sampling pass");
    if (n_events < 0 || gen_id >= 0x8000u) return fail(c, VAMP_ERR_INVALID_ARG, "bad n_events or gen_id");
    if (n_events > 0 && (!dev_records || ((uintptr_t)dev_records & 7u)))
        return fail(c, VAMP_ERR_INVALID_ARG, "dev_records must be non-NULL and 8-byte aligned");
    DeviceGuard g(c->dev);
    const int rec = (int)vamp_record_bytes(c->d);
    const int64_t B = c->gen_batch;
    const int64_t chunk = (int64_t)vamp::PASS_THREADS * c->var->cpt;
    const int64_t nchunks = (B + chunk - 1) / chunk;
    if (c->g_cap < nchunks * chunk) {
        cudaFree(c->g_staging); cudaFree(c->g_callidx); cudaFree(c->g_counts); cudaFree(c->g_offsets);
        c->g_staging = nullptr; c->g_callidx = nullptr; c->g_counts = nullptr; c->g_offsets = nullptr;
        c->g_cap = 0;
        const int64_t slots = nchunks * chunk;
        if (cudaMalloc(&c->g_staging, (size_t)slots * rec) != cudaSuccess ||
            cudaMalloc(&c->g_callidx, (size_t)slots * 4) != cudaSuccess ||
            cudaMalloc(&c->g_counts, (size_t)nchunks * 4) != cudaSuccess ||
            cudaMalloc(&c->g_offsets, (size_t)nchunks * 8) != cudaSuccess)
            return fail(c, VAMP_ERR_OOM, "generation staging allocation failed");
        c->g_cap = slots;
    }
    VAMP_CK(c, vamp::launch_gen_prepare(c->prm, c->stream));
    vamp::PassArgs G = pass_args(c, 0);
    G.rec_bytes = rec;
    G.batch = B;
    G.chunk = chunk;
    G.nchunks = nchunks;
    G.staging = c->g_staging;
    G.callidx = c->g_callidx;
    G.counts = c->g_counts;
    G.offsets = c->g_offsets;
    const int grid = (int)std::min<int64_t>(nchunks, c->grid_gen);
    int64_t written = 0, used = 0, over = 0;
    uint32_t b = 0;
    vamp_status st = VAMP_OK;
    while (written < n_events) {
        if (b >= 0x10000u) { st = fail(c, VAMP_ERR_TIMEOUT, "65536 generation batches did not yield n_events"); break; }
        G.field = 0x80000000u | (gen_id << 16) | b;
        unsigned char* outp = (unsigned char*)dev_records + written * rec;
        if (c->prof) VAMP_CK(c, cudaEventRecord(c->ev[0], c->stream));
        VAMP_CK(c, c->var->launch(c->prm, 1, G, grid, c->smem_gen, c->stream));
        if (c->prof) VAMP_CK(c, cudaEventRecord(c->ev[1], c->stream));
        VAMP_CK(c, vamp::launch_gen_finish(c->prm, G, n_events - written, outp, c->stream));
        st = read_head(c);
        if (st != VAMP_OK) return st;
        if (c->prof) {
            float ms = 0.f;
            VAMP_CK(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
            c->prof_gen_ms += ms;
            c->prof_gen_n += 1;
        }
        written += c->h_head->gen_take;
        used += c->h_head->gen_used;
        over += c->h_head->gen_over;
        ++b;
    }
    if (n_written) *n_written = written;
    if (n_calls_used) *n_calls_used = used;
    if (n_overweight) *n_overweight = over;
    if (st != VAMP_OK) return st;
    st = read_head(c);
    if (st != VAMP_OK) return st;
    return take_numeric_flag(c);
}

vamp_status vamp_get_state(vamp_ctx* c, double* edges, double* alpha, double* shift, double* w_max)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    DeviceGuard g(c->dev);
    const size_t rows = (size_t)c->K * c->d;
    if (edges) VAMP_CK(c, cudaMemcpyAsync(edges, c->prm.edges64, rows * (c->n + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    if (alpha) VAMP_CK(c, cudaMemcpyAsync(alpha, c->prm.alpha, c->K * 8, cudaMemcpyDeviceToHost, c->stream));
    if (shift) VAMP_CK(c, cudaMemcpyAsync(shift, c->prm.shift, c->K * 8, cudaMemcpyDeviceToHost, c->stream));
    vamp_status s = read_head(c);
    if (s != VAMP_OK) return s;
    if (w_max) *w_max = c->h_head->wmax_gen;
    return VAMP_OK;
}

vamp_status vamp_set_state(vamp_ctx* c, const double* edges, const double* alpha, const double* shift, double w_max)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    const size_t rows = (size_t)c->K * c->d;
    const int n = c->n;
    if (edges) {
        for (size_t r = 0; r < rows; ++r) {
            const double* e = edges + r * (n + 1);
            if (e[0] != 0.0 || e[n] != 1.0) return fail(c, VAMP_ERR_INVALID_ARG, "grid rows must run from 0 to 1");
            for (int j = 0; j < n; ++j)
                if (!(e[j + 1] > e[j])) return fail(c, VAMP_ERR_INVALID_ARG, "grid edges must increase strictly");
        }
    }
    if (alpha) {
        double s = 0.0;
        for (int q = 0; q < c->K; ++q) {
            if (!(alpha[q] >= 0.0) || !std::isfinite(alpha[q])) return fail(c, VAMP_ERR_INVALID_ARG, "alpha must be >= 0");
            s += alpha[q];
        }
        if (!(s > 0.0)) return fail(c, VAMP_ERR_INVALID_ARG, "alpha must not sum to 0");
    }
    if (!(w_max >= 0.0) || !std::isfinite(w_max)) return fail(c, VAMP_ERR_INVALID_ARG, "w_max must be finite and >= 0");
    DeviceGuard g(c->dev);
    if (edges) VAMP_CK(c, cudaMemcpyAsync(c->prm.edges64, edges, rows * (n + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    if (alpha) VAMP_CK(c, cudaMemcpyAsync(c->prm.alpha, alpha, c->K * 8, cudaMemcpyHostToDevice, c->stream));
    if (shift) VAMP_CK(c, cudaMemcpyAsync(c->prm.shift, shift, c->K * 8, cudaMemcpyHostToDevice, c->stream));
    VAMP_CK(c, cudaMemcpyAsync(&c->prm.sc->wmax_gen, &w_max, 8, cudaMemcpyHostToDevice, c->stream));
    VAMP_CK(c, vamp::launch_derive(c->prm, c->stream));
    if (c->uni_on) VAMP_CK(c, vamp::launch_union_build(c->prm, c->stream));
    VAMP_CK(c, cudaStreamSynchronize(c->stream));
    c->have_pass = 1;
    return VAMP_OK;
}

// ---- checkpoint / restore ----------------------------------------------------
namespace {
constexpr char CKP_MAGIC[8] = {'V', 'A', 'M', 'P', 'C', 'K', 'P', '1'};
struct CkpHeader {
    char magic[8];
    int32_t d, K, n, precision;
    int32_t n_hist, pad;
    double w_max;
};
size_t ckp_bytes(int d, int K, int n, int n_hist)
{
    const size_t edges = (size_t)K * d * (n + 1);
    return sizeof(CkpHeader) + 8 * (edges + 2 * (size_t)K + 2 * (size_t)n_hist) + 8 * (((size_t)n_hist * 4 + 7) / 8);
}
}  // namespace

int64_t vamp_checkpoint_bytes(vamp_ctx* c)
{
    if (!c) return -1;
    if (read_head(c) != VAMP_OK) return -1;
    return (int64_t)ckp_bytes(c->d, c->K, c->n, c->h_head->n_hist);
}

vamp_status vamp_checkpoint(vamp_ctx* c, void* host_buf, int64_t bytes)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!host_buf) return fail(c, VAMP_ERR_INVALID_ARG, "host_buf is required");
    DeviceGuard g(c->dev);
    vamp_status s = read_head(c);
    if (s != VAMP_OK) return s;
    const int nh = c->h_head->n_hist;
    if (bytes < (int64_t)ckp_bytes(c->d, c->K, c->n, nh)) return fail(c, VAMP_ERR_INVALID_ARG, "buffer too small");
    CkpHeader h{};
    std::memcpy(h.magic, CKP_MAGIC, 8);
    h.d = c->d;
    h.K = c->K;
    h.n = c->n;
    h.precision = c->fp32 ? VAMP_PREC_FP32_EVAL : VAMP_PREC_FP64;
    h.n_hist = nh;
    h.w_max = c->h_head->wmax_gen;
    unsigned char* o = static_cast<unsigned char*>(host_buf);
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    const size_t ne = (size_t)c->K * c->d * (c->n + 1);
    const Params& P = c->prm;
    VAMP_CK(c, cudaMemcpyAsync(o, P.edges64, ne * 8, cudaMemcpyDeviceToHost, c->stream));
    o += ne * 8;
    VAMP_CK(c, cudaMemcpyAsync(o, P.alpha, (size_t)c->K * 8, cudaMemcpyDeviceToHost, c->stream));
    o += (size_t)c->K * 8;
    VAMP_CK(c, cudaMemcpyAsync(o, P.shift, (size_t)c->K * 8, cudaMemcpyDeviceToHost, c->stream));
    o += (size_t)c->K * 8;
    if (nh > 0) {
        VAMP_CK(c, cudaMemcpyAsync(o, P.sc->hist_I, (size_t)nh * 8, cudaMemcpyDeviceToHost, c->stream));
        o += (size_t)nh * 8;
        VAMP_CK(c, cudaMemcpyAsync(o, P.sc->hist_V, (size_t)nh * 8, cudaMemcpyDeviceToHost, c->stream));
        o += (size_t)nh * 8;
        VAMP_CK(c, cudaMemcpyAsync(o, P.sc->hist_comb, (size_t)nh * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    VAMP_CK(c, cudaStreamSynchronize(c->stream));
    return VAMP_OK;
}

vamp_status vamp_restore(vamp_ctx* c, const void* host_buf, int64_t bytes)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!host_buf || bytes < (int64_t)sizeof(CkpHeader)) return fail(c, VAMP_ERR_INVALID_ARG, "no checkpoint");
    CkpHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    if (std::memcmp(h.magic, CKP_MAGIC, 8) != 0) return fail(c, VAMP_ERR_INVALID_ARG, "not a checkpoint");
    if (h.d != c->d || h.K != c->K || h.n != c->n)
        return fail(c, VAMP_ERR_INVALID_ARG, "checkpoint of another shape (d, K, n)");
    if (h.n_hist < 0 || h.n_hist > 1024 || bytes < (int64_t)ckp_bytes(h.d, h.K, h.n, h.n_hist))
        return fail(c, VAMP_ERR_INVALID_ARG, "truncated checkpoint");
    const unsigned char* o = static_cast<const unsigned char*>(host_buf) + sizeof h;
    const size_t ne = (size_t)c->K * c->d * (c->n + 1);
    std::vector<double> edges(ne), alpha(c->K), shift(c->K);
    std::memcpy(edges.data(), o, ne * 8);
    o += ne * 8;
    std::memcpy(alpha.data(), o, (size_t)c->K * 8);
    o += (size_t)c->K * 8;
    std::memcpy(shift.data(), o, (size_t)c->K * 8);
    o += (size_t)c->K * 8;
    // grids, α, shifts and w_max through the validating state upload
    vamp_status s = vamp_set_state(c, edges.data(), alpha.data(), shift.data(), h.w_max);
    if (s != VAMP_OK) return s;
    DeviceGuard g(c->dev);
    const Params& P = c->prm;
    if (h.n_hist > 0) {
        VAMP_CK(c, cudaMemcpyAsync(P.sc->hist_I, o, (size_t)h.n_hist * 8, cudaMemcpyHostToDevice, c->stream));
        o += (size_t)h.n_hist * 8;
        VAMP_CK(c, cudaMemcpyAsync(P.sc->hist_V, o, (size_t)h.n_hist * 8, cudaMemcpyHostToDevice, c->stream));
        o += (size_t)h.n_hist * 8;
        VAMP_CK(c, cudaMemcpyAsync(P.sc->hist_comb, o, (size_t)h.n_hist * 4, cudaMemcpyHostToDevice, c->stream));
    }
    const int32_t nh = h.n_hist;
    VAMP_CK(c, cudaMemcpyAsync(&P.sc->n_hist, &nh, sizeof nh, cudaMemcpyHostToDevice, c->stream));
    VAMP_CK(c, cudaStreamSynchronize(c->stream));
    return VAMP_OK;
}

vamp_status vamp_get_pass(vamp_ctx* c, double* D, double* Ic, double* Vc, int64_t* Nc)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    DeviceGuard g(c->dev);
    const size_t rows = (size_t)c->K * c->d;
    if (D) VAMP_CK(c, cudaMemcpyAsync(D, c->prm.D, rows * c->n * 8, cudaMemcpyDeviceToHost, c->stream));
    if (Ic) VAMP_CK(c, cudaMemcpyAsync(Ic, c->prm.Ic, c->K * 8, cudaMemcpyDeviceToHost, c->stream));
    if (Vc) VAMP_CK(c, cudaMemcpyAsync(Vc, c->prm.Vc, c->K * 8, cudaMemcpyDeviceToHost, c->stream));
    if (Nc) VAMP_CK(c, cudaMemcpyAsync(Nc, c->prm.Nc, c->K * 8, cudaMemcpyDeviceToHost, c->stream));
    VAMP_CK(c, cudaStreamSynchronize(c->stream));
    return VAMP_OK;
}

vamp_status vamp_eval_calls(vamp_ctx* c, int32_t mode, uint32_t field, uint32_t call0, int32_t count, double* x,
                            double* p, int32_t* jf, int32_t* bins, double* fgwc)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (count < 0 || (mode != 0 && mode != 1) || !fgwc) return fail(c, VAMP_ERR_INVALID_ARG, "bad eval arguments");
    if (count == 0) return VAMP_OK;
    if (mode == 0 && field >= 0x80000000u) return fail(c, VAMP_ERR_INVALID_ARG, "integration field must be < 2^31");
    DeviceGuard g(c->dev);
    if (mode == 0) {
        vamp_status s = read_head(c);
        if (s != VAMP_OK) return s;
        if ((int64_t)call0 + count > c->h_head->n_total)
            return fail(c, VAMP_ERR_INVALID_ARG, "calls beyond the current allocation");
    } else {
        VAMP_CK(c, vamp::launch_gen_prepare(c->prm, c->stream));
    }
    const int d = c->d, K = c->K;
    const size_t nx = (size_t)count * d, nb = (size_t)count * K * d;
    void* buf = nullptr;
    const size_t bytes = nx * 8 * 2 + nx * 4 + nb * 4 + (size_t)count * 4 * 8 + 1024;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return fail(c, VAMP_ERR_OOM, "eval buffer allocation failed");
    auto a256 = [](size_t v) { return (v + 255) & ~size_t(255); };
    char* q = (char*)buf;
    vamp::EvalArgs A{};
    A.mode = mode; A.field = field; A.call0 = call0; A.count = count;
    A.x = (double*)q; q += a256(nx * 8);
    A.p = (double*)q; q += a256(nx * 8);
    A.jf = (int*)q; q += a256(nx * 4);
    A.fgwc = (double*)q; q += a256((size_t)count * 32);
    A.bins = (int*)q;
    vamp_status st = VAMP_OK;
    cudaError_t e = vamp::launch_eval(c->prm, c->fp32, A, c->stream);
    if (e == cudaSuccess && x) e = cudaMemcpyAsync(x, A.x, nx * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, A.p, nx * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && jf) e = cudaMemcpyAsync(jf, A.jf, nx * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && bins) e = cudaMemcpyAsync(bins, A.bins, nb * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fgwc, A.fgwc, (size_t)count * 32, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = cuda_fail(c, e, "vamp_eval_calls");
    cudaFree(buf);
    return st;
}

vamp_status vamp_profile(vamp_ctx* c, int32_t enable)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    DeviceGuard g(c->dev);
    if (enable && !c->ev[0]) {
        VAMP_CK(c, cudaEventCreate(&c->ev[0]));
        VAMP_CK(c, cudaEventCreate(&c->ev[1]));
    }
    c->prof = enable ? 1 : 0;
    c->prof_sample_ms = c->prof_gen_ms = 0.0;
    c->prof_sample_n = c->prof_gen_n = 0;
    if (!c->prof_pending.empty()) VAMP_CK(c, cudaStreamSynchronize(c->stream));
    for (auto& pr : c->prof_pending) { c->ev_pool.push_back(pr.first); c->ev_pool.push_back(pr.second); }
    c->prof_pending.clear();
    return VAMP_OK;
}

vamp_status vamp_kernel_stats(vamp_ctx* c, double* sample_ms, int64_t* sample_launches, double* gen_ms,
                              int64_t* gen_launches)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!c->prof_pending.empty()) {
        DeviceGuard g(c->dev);
        VAMP_CK(c, cudaStreamSynchronize(c->stream));
        for (auto& pr : c->prof_pending) {
            float ms = 0.f;
            VAMP_CK(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
            c->prof_sample_ms += ms;
            c->prof_sample_n += 1;
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        c->prof_pending.clear();
    }
    if (sample_ms) *sample_ms = c->prof_sample_ms;
    if (sample_launches) *sample_launches = c->prof_sample_n;
    if (gen_ms) *gen_ms = c->prof_gen_ms;
    if (gen_launches) *gen_launches = c->prof_gen_n;
    return VAMP_OK;
}

vamp_status vamp_pass_kernel_info(const vamp_ctx* c, int32_t* fp32, int32_t* cpt, int32_t* shape_d,
                                  int32_t* shape_n, int32_t* ctas_per_sm)
{
    if (!c || !c->var) return VAMP_ERR_INVALID_ARG;
    if (fp32) *fp32 = c->var->fp32;
    if (cpt) *cpt = c->var->cpt;
    if (shape_d) *shape_d = c->var->D;
    if (shape_n) *shape_n = c->var->NB;
    if (ctas_per_sm) *ctas_per_sm = c->var->minb;
    return VAMP_OK;
}

vamp_status vamp_pass_kernel_name(const vamp_ctx* c, int32_t mode, char* buf, int32_t len)
{
    if (!c || !c->var || (mode != 0 && mode != 1) || !buf || len < 1) return VAMP_ERR_INVALID_ARG;
    const vamp::PassVariant* v = c->var;
    const int k = std::snprintf(buf, (size_t)len, "%s<%s, %d, %d, %d, %d, %d>", v->family,
                                v->fp32 ? "float" : "double", mode, v->cpt, v->D, v->NB, v->minb);
    return (k < 0 || k >= len) ? VAMP_ERR_INVALID_ARG : VAMP_OK;
}

vamp_status vamp_pass_kernel_candidates(const vamp_ctx* c, int32_t* count)
{
    if (!c || !count) return VAMP_ERR_INVALID_ARG;
    *count = (int32_t)candidates_of(c).size();
    return VAMP_OK;
}

vamp_status vamp_select_pass_kernel(vamp_ctx* c, int32_t index)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    const std::vector<const PassVariant*> cand = candidates_of(c);
    if (index < 0 || index >= (int32_t)cand.size()) return fail(c, VAMP_ERR_INVALID_ARG, "no such pass-kernel candidate");
    DeviceGuard g(c->dev);
    const vamp_status s = use_variant(c, cand[index]);
    if (s != VAMP_OK) return s;
    c->tuned = 1;  // the autotuner leaves a pinned choice alone
    return VAMP_OK;
}

vamp_status vamp_selftest_bounded_wait(int64_t limit_cycles, int64_t* waited_cycles)
{
    if (limit_cycles < 1 || limit_cycles > (int64_t(1) << 31)) return VAMP_ERR_INVALID_ARG;
    void* mem = nullptr;
    if (cudaMalloc(&mem, 16) != cudaSuccess) return VAMP_ERR_OOM;
    unsigned int* flag = static_cast<unsigned int*>(mem);
    long long* cycles = reinterpret_cast<long long*>(static_cast<unsigned char*>(mem) + 8);
    unsigned int h_flag = 0;
    long long h_cycles = 0;
    cudaError_t e = cudaMemset(mem, 0, 16);
    if (e == cudaSuccess) e = vamp::launch_wait_selftest((long long)limit_cycles, flag, cycles, 0);
    if (e == cudaSuccess) e = cudaMemcpy(&h_flag, flag, sizeof h_flag, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&h_cycles, cycles, sizeof h_cycles, cudaMemcpyDeviceToHost);
    cudaFree(mem);
    if (e != cudaSuccess) return VAMP_ERR_CUDA;
    if (waited_cycles) *waited_cycles = h_cycles;
    return (h_flag & vamp::ERR_TIMEOUT) ? VAMP_ERR_TIMEOUT : VAMP_OK;
}

}  // extern "C"

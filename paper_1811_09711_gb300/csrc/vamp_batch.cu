// vamp_batch.cu -- many independent integrations advanced together: one
// persistent pass kernel over all instances per iteration, the small steps
// as a handful of multi-instance kernels, and the whole iteration captured
// once as a CUDA graph and replayed (its per-iteration arguments -- calls per
// instance, iteration index, adaptation flags -- are copied from pinned host
// memory by the graph's first nodes).
#include "../../include/vamp.h"
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using vamp::Params;
using vamp::Scalars;

struct vamp_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;   // owned
    int n = 0, fp32 = 0;
    std::vector<Params> prm;
    std::vector<int> tiles, combine_from, pair_off, row_off, K, d, nb;
    std::vector<size_t> S;          // lookup-block bytes per instance (evaluation precision)
    int npairs = 0, nrows = 0, max_n = 0, sm_count = 0;
    void* arena = nullptr;
    // device arrays
    Params* d_inst = nullptr;
    int* d_tiles = nullptr;
    int* d_comb = nullptr;
    int64_t* d_ncalls = nullptr;
    uint32_t* d_iter = nullptr;
    int* d_pair_off = nullptr;
    long long* d_pair_prefix = nullptr;
    int* d_row_off = nullptr;
    vamp::BatchCtl* d_ctl = nullptr;
    vamp::BatchIter* d_it = nullptr;
    double* d_results = nullptr;
    // pinned host mirrors
    vamp::BatchIter* h_it = nullptr;
    int64_t* h_ncalls = nullptr;
    uint32_t* h_iter = nullptr;
    double* h_results = nullptr;
    // launch shape
    int64_t item_calls = 0;
    int budget_kb = 112;
    int minb = 2;                   // CTAs per SM of the multi-instance kernel in use
    size_t smem = 0;
    int grid = 0;
    int tune = 1, tuned = 0;
    double tuned_ms = 0.0, fixed_ms = 0.0;
    int64_t fixed_item_calls = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // pseudo-stratified instances: cell sums per instance, sized by the calls
    // requested (grown between iterations; the kernels read the pointer from
    // the device parameter table, so the captured graph stays valid)
    int strat = 0;
    std::vector<double*> cellbuf;
    std::vector<int64_t> cellcap;
    std::string err;
};

namespace {

vamp_status bfail(vamp_batch* b, vamp_status s, const std::string& msg)
{
    if (b) b->err = msg;
    return s;
}

#define BCK(b, call)                                                                         \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return bfail((b), VAMP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Calls per thread of the multi-instance kernel's small-d classes: work
// items are sized in multiples of PASS_THREADS times this.
int calls_per_thread(int) { return 2; }

vamp::MultiArgs margs(const vamp_batch* b)
{
    vamp::MultiArgs M{};
    M.inst = b->d_inst;
    M.tiles = b->d_tiles;
    M.combine_from = b->d_comb;
    M.ncalls = b->d_ncalls;
    M.iter = b->d_iter;
    M.pair_off = b->d_pair_off;
    M.pair_prefix = b->d_pair_prefix;
    M.row_off = b->d_row_off;
    M.ctl = b->d_ctl;
    M.it = b->d_it;
    M.results = b->d_results;
    M.n_inst = b->n;
    M.npairs = b->npairs;
    M.nrows = b->nrows;
    M.max_n = b->max_n;
    M.item_calls = b->item_calls;
    M.any_strat = b->strat;
    return M;
}

// Tiles and shared memory for a budget (KB) of the multi-instance kernel.
vamp_status apply_shape(vamp_batch* b, int budget_kb, int64_t item_calls)
{
    const size_t budget = (size_t)budget_kb * 1024;
    b->minb = budget_kb > 80 ? 2 : 3;  // 112 KB: two CTAs per SM; 72 KB: three
    size_t smem = 0;
    for (int i = 0; i < b->n; ++i) {
        const size_t ds = (size_t)b->d[i] * b->nb[i] * 8;
        const size_t fixed = vamp::SMEM_HEAD + vamp::PARAMS_SLOT + ds;
        long t = budget > fixed ? (long)((budget - fixed) / (2 * b->S[i])) : 1;
        if (t < 1) t = 1;
        if (t > b->K[i]) t = b->K[i];
        b->tiles[i] = (int)t;
        smem = std::max(smem, fixed + 2 * (size_t)t * b->S[i]);
    }
    int maxsm = 0;
    BCK(b, cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->dev));
    if ((int)smem > maxsm) return bfail(b, VAMP_ERR_INVALID_ARG, "an instance's grid is too large for shared memory");
    BCK(b, vamp::ensure_smem(vamp::pass_multi_kernel(b->fp32, b->minb, b->strat), smem));
    int bps = 0;
    BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, vamp::pass_multi_kernel(b->fp32, b->minb, b->strat),
                                                         vamp::PASS_THREADS,
                                                         smem));
    BCK(b, cudaMemcpyAsync(b->d_tiles, b->tiles.data(), b->n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    b->smem = smem;
    b->grid = (bps > 0 ? bps : 1) * b->sm_count;
    b->budget_kb = budget_kb;
    b->item_calls = item_calls;
    return VAMP_OK;
}

// Cell-sum buffers of the pseudo-stratified instances for a pass of n_calls
// each: at most (N + K n_min) / 2 + K cells (two calls or more per cell).
vamp_status ensure_cells(vamp_batch* b, const int64_t* n_calls)
{
    for (int i = 0; i < b->n; ++i) {
        Params& P = b->prm[i];
        if (!P.stratified) continue;
        const int64_t need = (n_calls[i] + (int64_t)P.K * P.n_min) / 2 + P.K;
        if (need <= b->cellcap[i]) continue;
        BCK(b, cudaStreamSynchronize(b->stream));
        cudaFree(b->cellbuf[i]);
        b->cellbuf[i] = nullptr;
        b->cellcap[i] = 0;
        P.cellsum = nullptr;
        if (cudaMalloc(&b->cellbuf[i], (size_t)need * 8) != cudaSuccess) {
            b->cellbuf[i] = nullptr;
            return bfail(b, VAMP_ERR_OOM, "cell sums of a pseudo-stratified instance");
        }
        b->cellcap[i] = need;
        P.cellsum = b->cellbuf[i];
        BCK(b, cudaMemcpyAsync(b->d_inst + i, &P, sizeof(Params), cudaMemcpyHostToDevice, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
    }
    return VAMP_OK;
}

void drop_graph(vamp_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Enqueues one iteration (arguments already in the pinned mirrors).
vamp_status enqueue_iteration(vamp_batch* b, bool pass_only)
{
    BCK(b, cudaMemcpyAsync(b->d_it, b->h_it, sizeof(vamp::BatchIter), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_ncalls, b->h_ncalls, b->n * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_iter, b->h_iter, b->n * sizeof(uint32_t), cudaMemcpyHostToDevice, b->stream));
    const vamp::MultiArgs M = margs(b);
    BCK(b, vamp::launch_batch_begin(M, b->stream));
    BCK(b, vamp::launch_pass_multi(b->fp32, b->minb, M, b->grid, b->smem, b->stream));
    if (pass_only) return VAMP_OK;
    BCK(b, vamp::launch_batch_after(M, b->stream));
    BCK(b, cudaMemcpyAsync(b->h_results, b->d_results, (size_t)b->n * 9 * sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream));
    return VAMP_OK;
}

// Autotuner: times the pass of one iteration at the requested calls (once
// per shape after a warm-up launch) for work-item sizes x shared-memory
// budgets and keeps the fastest; the fixed shape (one batch per item,
// 112 KB) is timed too, for reference.
vamp_status autotune(vamp_batch* b, const int64_t* n_calls)
{
    const int64_t B = (int64_t)vamp::PASS_THREADS * calls_per_thread(b->fp32);
    for (int i = 0; i < b->n; ++i) b->h_ncalls[i] = n_calls[i];
    b->h_it->iteration = 0x7fffffffu;
    b->h_it->adapt = 0;
    for (int i = 0; i < b->n; ++i) b->h_iter[i] = 0x7fffffffu;
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    const int budgets[2] = {112, 72};
    const int64_t mults[5] = {1, 2, 4, 8, 16};
    float best = 1e30f;
    int best_budget = 112;
    int64_t best_items = B;
    for (int bi = 0; bi < 2; ++bi) {
        for (int mi = 0; mi < 5; ++mi) {
            vamp_status st = apply_shape(b, budgets[bi], B * mults[mi]);
            if (st != VAMP_OK) return st;
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                BCK(b, cudaEventRecord(e0, b->stream));
                st = enqueue_iteration(b, true);
                if (st != VAMP_OK) return st;
                BCK(b, cudaEventRecord(e1, b->stream));
                BCK(b, cudaEventSynchronize(e1));
                BCK(b, cudaEventElapsedTime(&ms, e0, e1));
            }
            if (bi == 0 && mi == 0) b->fixed_ms = ms;
            if (ms < best) { best = ms; best_budget = budgets[bi]; best_items = B * mults[mi]; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned_ms = best;
    b->fixed_item_calls = B;
    // the probes left accumulators and maxima behind: the next iteration's
    // first kernel clears the accumulators; clear the per-instance scalars'
    // pass maxima and flags here
    for (int i = 0; i < b->n; ++i)
        BCK(b, cudaMemsetAsync(b->prm[i].sc, 0, offsetof(Scalars, gen_bmax_bits), b->stream));
    return apply_shape(b, best_budget, best_items);
}

}  // namespace

extern "C" {

const char* vamp_batch_last_error(const vamp_batch* b) { return b ? b->err.c_str() : ""; }

void vamp_batch_destroy(vamp_batch* b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->dev) cudaSetDevice(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (double* q : b->cellbuf) cudaFree(q);
    cudaFree(b->arena);
    cudaFreeHost(b->h_it);
    cudaFreeHost(b->h_ncalls);
    cudaFreeHost(b->h_iter);
    cudaFreeHost(b->h_results);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (prev >= 0 && prev != b->dev) cudaSetDevice(prev);
    delete b;
}

vamp_status vamp_batch_create(const vamp_config* cfgs, int32_t n, int32_t autotune_tiles, vamp_batch** out)
{
    if (!out) return VAMP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfgs || n < 1) return VAMP_ERR_INVALID_ARG;
    vamp_batch* b = new (std::nothrow) vamp_batch();
    if (!b) return VAMP_ERR_OOM;
    b->n = n;
    b->tune = autotune_tiles ? 1 : 0;
    std::vector<vamp::Setup> setups(n);
    std::vector<vamp::Arena> ars(n);
    b->prm.resize(n);
    b->cellbuf.assign(n, nullptr);
    b->cellcap.assign(n, 0);
    b->tiles.assign(n, 1);
    b->combine_from.resize(n);
    b->K.resize(n);
    b->d.resize(n);
    b->nb.resize(n);
    b->S.resize(n);
    b->pair_off.assign(n + 1, 0);
    b->row_off.assign(n + 1, 0);
    size_t total = 0;
    std::vector<size_t> offs(n);
    for (int i = 0; i < n; ++i) {
        std::string why;
        Params p{};
        if (!vamp::build_setup(&cfgs[i], p, setups[i], why)) {
            delete b;
            return VAMP_ERR_INVALID_ARG;
        }
        if (i == 0) b->fp32 = setups[0].fp32;
        if (setups[i].fp32 != b->fp32) { delete b; return VAMP_ERR_INVALID_ARG; }
        b->prm[i] = p;
        if (p.stratified) b->strat = 1;
        ars[i] = vamp::plan_arena(p);
        offs[i] = total;
        total += a256(ars[i].bytes);
        b->combine_from[i] = cfgs[i].combine_from;
        b->K[i] = p.K;
        b->d[i] = p.d;
        b->nb[i] = p.n;
        b->S[i] = (size_t)(b->fp32 ? p.lay32.bytes : p.lay64.bytes);
        b->pair_off[i + 1] = b->pair_off[i] + p.K;
        b->row_off[i + 1] = b->row_off[i] + p.K * p.d;
        b->max_n = std::max(b->max_n, p.n);
    }
    b->npairs = b->pair_off[n];
    b->nrows = b->row_off[n];
    // control arrays after the instances' arenas
    const size_t o_inst = total;
    total += a256((size_t)n * sizeof(Params));
    const size_t o_tiles = total;
    total += a256((size_t)n * 4);
    const size_t o_comb = total;
    total += a256((size_t)n * 4);
    const size_t o_nc = total;
    total += a256((size_t)n * 8);
    const size_t o_itr = total;
    total += a256((size_t)n * 4);
    const size_t o_po = total;
    total += a256((size_t)(n + 1) * 4);
    const size_t o_pp = total;
    total += a256((size_t)(b->npairs + 1) * 8);
    const size_t o_ro = total;
    total += a256((size_t)(n + 1) * 4);
    const size_t o_ctl = total;
    total += a256(sizeof(vamp::BatchCtl));
    const size_t o_it = total;
    total += a256(sizeof(vamp::BatchIter));
    const size_t o_res = total;
    total += a256((size_t)n * 9 * 8);

    vamp_status st = VAMP_OK;
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->arena, total);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_it, sizeof(vamp::BatchIter));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ncalls, (size_t)n * 8);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_iter, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_results, (size_t)n * 9 * 8);
    if (e != cudaSuccess) {
        vamp_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? VAMP_ERR_OOM : VAMP_ERR_CUDA;
    }
    unsigned char* base = (unsigned char*)b->arena;
    b->d_inst = (Params*)(base + o_inst);
    b->d_tiles = (int*)(base + o_tiles);
    b->d_comb = (int*)(base + o_comb);
    b->d_ncalls = (int64_t*)(base + o_nc);
    b->d_iter = (uint32_t*)(base + o_itr);
    b->d_pair_off = (int*)(base + o_po);
    b->d_pair_prefix = (long long*)(base + o_pp);
    b->d_row_off = (int*)(base + o_ro);
    b->d_ctl = (vamp::BatchCtl*)(base + o_ctl);
    b->d_it = (vamp::BatchIter*)(base + o_it);
    b->d_results = (double*)(base + o_res);
#define BCREATE(call)                                                                               \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) { st = bfail(b, VAMP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); goto fail; } \
    } while (0)
    BCREATE(cudaMemsetAsync(b->arena, 0, total, b->stream));
    for (int i = 0; i < n; ++i) {
        vamp::bind_arena(b->prm[i], base + offs[i], ars[i]);
        const Params& P = b->prm[i];
        const size_t rows = (size_t)P.K * P.d;
        std::vector<double> edges(rows * (P.n + 1)), alpha(P.K, 1.0 / (double)P.K);
        for (size_t r = 0; r < rows; ++r)
            for (int j = 0; j <= P.n; ++j) edges[r * (P.n + 1) + j] = (double)j / (double)P.n;
        BCREATE(cudaMemcpyAsync(P.edges64, edges.data(), edges.size() * 8, cudaMemcpyHostToDevice, b->stream));
        BCREATE(cudaMemcpyAsync(P.alpha, alpha.data(), P.K * 8, cudaMemcpyHostToDevice, b->stream));
        BCREATE(vamp::upload_setup(P, setups[i], b->stream));
        BCREATE(vamp::launch_derive(P, b->stream));
        BCREATE(cudaStreamSynchronize(b->stream));  // host vectors go out of scope
    }
    BCREATE(cudaMemcpyAsync(b->d_inst, b->prm.data(), (size_t)n * sizeof(Params), cudaMemcpyHostToDevice, b->stream));
    BCREATE(cudaMemcpyAsync(b->d_comb, b->combine_from.data(), (size_t)n * 4, cudaMemcpyHostToDevice, b->stream));
    BCREATE(cudaMemcpyAsync(b->d_pair_off, b->pair_off.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, b->stream));
    BCREATE(cudaMemcpyAsync(b->d_row_off, b->row_off.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, b->stream));
    BCREATE(cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->dev));
    BCREATE(cudaStreamSynchronize(b->stream));
#undef BCREATE
    st = apply_shape(b, 112, (int64_t)vamp::PASS_THREADS * calls_per_thread(b->fp32));
    if (st != VAMP_OK) goto fail;
    b->fixed_item_calls = b->item_calls;
    *out = b;
    return VAMP_OK;
fail:
    vamp_batch_destroy(b);
    return st;
}

vamp_status vamp_batch_iterate(vamp_batch* b, const int64_t* n_calls, uint32_t iteration, int32_t adapt,
                               vamp_pass_result* results)
{
    if (!b) return VAMP_ERR_INVALID_ARG;
    if (!n_calls || !results) return bfail(b, VAMP_ERR_INVALID_ARG, "n_calls and results are required");
    if (iteration >= 0x80000000u) return bfail(b, VAMP_ERR_INVALID_ARG, "iteration must be < 2^31");
    for (int i = 0; i < b->n; ++i)
        if (n_calls[i] < 1 || n_calls[i] > int64_t(0xffffffff) ||
            n_calls[i] > int64_t(0xffffffff) - (int64_t)b->K[i] * b->prm[i].n_min)
            return bfail(b, VAMP_ERR_INVALID_ARG, "calls per instance must be >= 1 and < 2^32");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->dev) cudaSetDevice(b->dev);
    vamp_status st = ensure_cells(b, n_calls);
    if (st == VAMP_OK && b->tune && !b->tuned) {
        st = autotune(b, n_calls);
        b->tuned = 1;
        drop_graph(b);
    }
    if (st == VAMP_OK) {
        for (int i = 0; i < b->n; ++i) {
            b->h_ncalls[i] = n_calls[i];
            b->h_iter[i] = iteration;
        }
        b->h_it->iteration = iteration;
        b->h_it->adapt = adapt;
        if (!b->exec) {
            cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                st = enqueue_iteration(b, false);
                cudaGraph_t g = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                if (st == VAMP_OK && e2 == cudaSuccess) {
                    b->graph = g;
                    e = cudaGraphInstantiate(&b->exec, g, 0);
                } else {
                    if (g) cudaGraphDestroy(g);
                    if (st == VAMP_OK) st = bfail(b, VAMP_ERR_CUDA, "graph capture failed");
                }
            }
            if (st == VAMP_OK && e != cudaSuccess) st = bfail(b, VAMP_ERR_CUDA, cudaGetErrorString(e));
        }
        if (st == VAMP_OK) {
            cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) st = bfail(b, VAMP_ERR_CUDA, std::string("iteration graph: ") + cudaGetErrorString(e));
        }
    }
    if (st == VAMP_OK) {
        unsigned flags = 0;
        for (int i = 0; i < b->n; ++i) {
            const double* r = b->h_results + (size_t)i * 9;
            results[i].integral = r[0];
            results[i].variance = r[1];
            results[i].w_max = r[2];
            results[i].efficiency = r[3];
            results[i].n_calls = (int64_t)r[4];
            results[i].combined = r[5];
            results[i].combined_sigma = r[6];
            results[i].chi2_dof = r[7];
            const unsigned f = (unsigned)r[8];
            if (f) {
                flags |= f;
                cudaMemsetAsync(&b->prm[i].sc->err, 0, sizeof(unsigned), b->stream);
            }
        }
        if (flags) {
            cudaStreamSynchronize(b->stream);
            st = (flags & vamp::ERR_TIMEOUT) ? bfail(b, VAMP_ERR_TIMEOUT, "a bounded wait gave up")
                                             : bfail(b, VAMP_ERR_NUMERIC, "a non-finite weight was produced");
        }
    }
    if (prev >= 0 && prev != b->dev) cudaSetDevice(prev);
    return st;
}

vamp_status vamp_batch_get_state(vamp_batch* b, int32_t instance, double* edges, double* alpha, double* shift,
                                 double* w_max)
{
    if (!b || instance < 0 || instance >= b->n) return VAMP_ERR_INVALID_ARG;
    const Params& P = b->prm[instance];
    const size_t rows = (size_t)P.K * P.d;
    if (edges) BCK(b, cudaMemcpyAsync(edges, P.edges64, rows * (P.n + 1) * 8, cudaMemcpyDeviceToHost, b->stream));
    if (alpha) BCK(b, cudaMemcpyAsync(alpha, P.alpha, P.K * 8, cudaMemcpyDeviceToHost, b->stream));
    if (shift) BCK(b, cudaMemcpyAsync(shift, P.shift, P.K * 8, cudaMemcpyDeviceToHost, b->stream));
    if (w_max) BCK(b, cudaMemcpyAsync(w_max, &P.sc->wmax_gen, 8, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return VAMP_OK;
}

vamp_status vamp_batch_tuning(const vamp_batch* b, int64_t* item_calls, int32_t* budget_kb, double* tuned_ms,
                              double* fixed_ms)
{
    if (!b) return VAMP_ERR_INVALID_ARG;
    if (item_calls) *item_calls = b->item_calls;
    if (budget_kb) *budget_kb = b->budget_kb;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    if (fixed_ms) *fixed_ms = b->fixed_ms;
    return VAMP_OK;
}

}  // extern "C"

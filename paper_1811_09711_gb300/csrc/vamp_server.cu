// vamp_server.cu -- continuous-batching request loop.
//
// Requests (integrate for a number of adaptation iterations, then generate
// unweighted events) are queued by vamp_server_submit and admitted by a
// scheduler thread into slots while the device-memory budget allows (the
// request's state arena and generation staging; the events go to the
// caller's buffer).  Every tick, all admitted requests that are
// still integrating advance one iteration together in ONE launch of the
// multi-instance pass kernel (plus the multi-instance allocation, result,
// rebinning and α kernels), each on its own random stream (its own iteration
// index); requests that reach their last iteration move to generation, whose
// batches run on per-request streams and overlap with the next ticks.  A
// request that arrives while others are on the GPU joins the next tick.
// Grids, α and running maxima stay resident on the device for the whole life
// of a request.  Latency = arrival to completion.
//
// Nothing on the request path synchronises the device: request memory comes
// from the server's own stream-ordered pool (cudaMallocFromPoolAsync /
// cudaFreeAsync on the request's stream), and the request's stream, event
// and pinned status slot are taken from a pool of lanes and given back.
#include "../../include/vamp.h"
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

using vamp::Params;
using vamp::Scalars;

namespace {

using clk = std::chrono::steady_clock;

double secs(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Req {
    uint64_t id = 0;
    // owned copy of the description
    vamp_config cfg{};
    std::vector<vamp_map_desc> ch, pk;
    std::vector<double> w;
    int iterations = 0;
    int64_t calls = 0, n_events = 0, max_gen_calls = 0;
    unsigned char* records = nullptr;   // caller's buffer
    double* state_out = nullptr;        // caller's buffer for the adapted state (optional)
    clk::time_point t_arrive, t_admit, t_done;
    // device state
    Params P{};
    vamp::Setup S;
    vamp::Arena ar{};
    void* mem = nullptr;
    size_t bytes = 0;
    unsigned char* staging = nullptr;
    uint32_t* callidx = nullptr;
    int* counts = nullptr;
    long long* offsets = nullptr;
    const vamp::PassVariant* var = nullptr;
    int tile = 1, grid_gen = 0;
    size_t smem_int = 0, smem_gen = 0;
    int64_t chunk = 0, nchunks = 0, gen_batch = 0;
    int lane = -1;             // index into the server's lanes
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Scalars* h_head = nullptr;
    // progress
    int phase = 0;  // 0 setting up, 1 integrating, 2 generating, 3 done
    bool in_tick = false;  // member of the multi-instance launch in flight
    int it_done = 0;
    int64_t calls_total = 0;
    vamp_pass_result last{};
    bool in_flight = false;
    uint32_t gen_b = 0;
    int64_t written = 0, used = 0, over = 0;
    vamp_status status = VAMP_OK;
};

}  // namespace

struct vamp_server {
    int dev = 0, fp32 = 1, max_slots = 0, sm_count = 0;
    int64_t budget = 0;
    std::atomic<int64_t> used_mem{0};
    std::atomic<int64_t> n_live{0};  // queued + active
    cudaStream_t stream = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> queue;
    std::vector<Req*> active;
    std::vector<vamp_request_result> done;
    bool stop = false;
    uint64_t next_id = 1;
    std::string err;
    // reusable per-request resources
    cudaMemPool_t pool = nullptr;
    struct Lane {
        cudaStream_t stream = nullptr;
        cudaEvent_t ev = nullptr;
    };
    std::vector<Lane> lanes;
    std::vector<int> free_lanes;
    unsigned char* h_heads = nullptr;  // pinned, one status slot per lane
    size_t head_stride = 0;
    // launch shape of the multi-instance kernel: three CTAs per SM with 72 KB
    // each in the FP32-eval form (the batch autotuner's usual pick for mixed
    // request shapes), two with 112 KB in FP64; cached per shared-memory size
    int tick_minb = 2;
    size_t tick_budget = vamp::TILE_BUDGET;
    size_t tick_smem = 0;
    int tick_grid = 0;
    int tick_strat = 0;                // kernel form of the cached shape: with the cell code
    cudaEvent_t tick_ev = nullptr;     // end of the launch in flight
    std::vector<Req*> tick_reqs;       // its members
    // multi-instance launch arrays (capacity grows on demand)
    void* marena = nullptr;
    size_t mcap_inst = 0, mcap_pairs = 0;
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
    void* hmem = nullptr;  // pinned mirrors
    Params* h_inst = nullptr;
    int* h_tiles = nullptr;
    int* h_comb = nullptr;
    int64_t* h_ncalls = nullptr;
    uint32_t* h_iter = nullptr;
    int* h_pair_off = nullptr;
    int* h_row_off = nullptr;
    vamp::BatchIter* h_it = nullptr;
    double* h_results = nullptr;
    // statistics
    std::atomic<int64_t> n_ticks{0}, calls_done{0}, events_done{0}, gen_batches{0};
    std::atomic<int32_t> n_queued{0}, n_integrating{0}, n_generating{0};
};

namespace {

// Takes a lane (stream, event, status slot), creating its stream and event
// on first use.  -1 if they cannot be created.
int take_lane(vamp_server* s)
{
    if (s->free_lanes.empty()) return -1;
    const int i = s->free_lanes.back();
    vamp_server::Lane& l = s->lanes[i];
    if (!l.stream && cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess) return -1;
    if (!l.ev && cudaEventCreateWithFlags(&l.ev, cudaEventDisableTiming) != cudaSuccess) return -1;
    s->free_lanes.pop_back();
    return i;
}

// Returns a request's memory to the pool (ordered after its work on its
// stream) and its lane to the free list; no device synchronisation.
void free_req(vamp_server* s, Req* r)
{
    if (r->mem) cudaFreeAsync(r->mem, r->stream);
    if (r->lane >= 0) s->free_lanes.push_back(r->lane);
    s->used_mem -= (int64_t)r->bytes;
    delete r;
}

// Bytes a request needs on the device once admitted: its state arena, the
// cell sums of a pseudo-stratified request (at most (N + K n_min) / 2 + K
// cells) and the generation staging of its pass kernel (chunks of
// PASS_THREADS * CPT calls).
size_t request_bytes(const Req* r, size_t* o_cells, size_t* o_stage, size_t* o_call, size_t* o_cnt, size_t* o_off)
{
    const int64_t chunk = (int64_t)vamp::PASS_THREADS * r->var->cpt;
    const int64_t B = r->cfg.gen_batch > 0 ? r->cfg.gen_batch : (int64_t(1) << 20);
    const int64_t nch = (B + chunk - 1) / chunk;
    const size_t rec = (size_t)vamp_record_bytes(r->cfg.d);
    const bool gen = r->n_events > 0;
    size_t off = a256(r->ar.bytes);
    *o_cells = off;
    if (r->P.stratified) off += a256((size_t)((r->calls + (int64_t)r->P.K * r->P.n_min) / 2 + r->P.K) * 8);
    *o_stage = off;
    off += gen ? a256((size_t)nch * chunk * rec) : 0;
    *o_call = off;
    off += gen ? a256((size_t)nch * chunk * 4) : 0;
    *o_cnt = off;
    off += gen ? a256((size_t)nch * 4) : 0;
    *o_off = off;
    off += gen ? a256((size_t)nch * 8) : 0;
    return off;
}

// Allocates an admitted request and enqueues its initialisation on its
// stream (uniform grids, α = 1/K, lookup blocks); the request joins the
// integration launches once the recorded event has completed.
vamp_status admit(vamp_server* s, Req* r)
{
    size_t o_cells, o_stage, o_call, o_cnt, o_off;
    r->lane = take_lane(s);
    if (r->lane < 0) return VAMP_ERR_CUDA;
    r->stream = s->lanes[r->lane].stream;
    r->ev = s->lanes[r->lane].ev;
    r->h_head = reinterpret_cast<Scalars*>(s->h_heads + (size_t)r->lane * s->head_stride);
    r->bytes = request_bytes(r, &o_cells, &o_stage, &o_call, &o_cnt, &o_off);
    cudaError_t e = cudaMallocFromPoolAsync(&r->mem, r->bytes, s->pool, r->stream);
    if (e != cudaSuccess) { r->mem = nullptr; r->bytes = 0; return VAMP_ERR_OOM; }
    s->used_mem += (int64_t)r->bytes;
    unsigned char* base = (unsigned char*)r->mem;
    vamp::bind_arena(r->P, base, r->ar);
    if (r->P.stratified) r->P.cellsum = reinterpret_cast<double*>(base + o_cells);
    r->staging = base + o_stage;
    r->callidx = (uint32_t*)(base + o_call);
    r->counts = (int*)(base + o_cnt);
    r->offsets = (long long*)(base + o_off);
    const Params& P = r->P;
    const size_t rows = (size_t)P.K * P.d;
    std::vector<double> edges(rows * (P.n + 1)), alpha(P.K, 1.0 / (double)P.K);
    for (size_t q = 0; q < rows; ++q)
        for (int j = 0; j <= P.n; ++j) edges[q * (P.n + 1) + j] = (double)j / (double)P.n;
    if (e == cudaSuccess) e = cudaMemsetAsync(r->mem, 0, r->ar.bytes, r->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.edges64, edges.data(), edges.size() * 8, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P.alpha, alpha.data(), P.K * 8, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) e = vamp::upload_setup(P, r->S, r->stream);
    if (e == cudaSuccess) e = vamp::launch_derive(P, r->stream);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, r->stream);  // setup done (polled)
    if (e != cudaSuccess) return VAMP_ERR_CUDA;
    // generation kernel of this shape
    vamp::pass_smem_for(P, s->fp32, r->var->minb, &r->tile, &r->smem_int, &r->smem_gen);
    e = vamp::ensure_smem(r->var->fn[1], r->smem_gen);
    int bps = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, r->var->fn[1], vamp::PASS_THREADS, r->smem_gen);
    if (e != cudaSuccess) return VAMP_ERR_CUDA;
    r->chunk = (int64_t)vamp::PASS_THREADS * r->var->cpt;
    r->gen_batch = r->cfg.gen_batch > 0 ? r->cfg.gen_batch : (int64_t(1) << 20);
    r->nchunks = (r->gen_batch + r->chunk - 1) / r->chunk;
    r->grid_gen = (int)std::min<int64_t>(r->nchunks, (int64_t)(bps > 0 ? bps : 1) * s->sm_count);
    r->t_admit = clk::now();
    r->phase = 0;
    r->in_flight = true;
    return VAMP_OK;
}

vamp_status grow_multi(vamp_server* s, size_t n, size_t npairs)
{
    if (n <= s->mcap_inst && npairs <= s->mcap_pairs) return VAMP_OK;
    const size_t ci = std::max(n, 2 * s->mcap_inst), cp = std::max(npairs, 2 * s->mcap_pairs);
    cudaFree(s->marena);
    cudaFreeHost(s->hmem);
    size_t off = 0;
    auto take = [&](size_t b) { const size_t o = off; off += a256(b); return o; };
    const size_t o_inst = take(ci * sizeof(Params)), o_tiles = take(ci * 4), o_comb = take(ci * 4),
                 o_nc = take(ci * 8), o_it2 = take(ci * 4), o_po = take((ci + 1) * 4), o_pp = take((cp + 1) * 8),
                 o_ro = take((ci + 1) * 4), o_ctl = take(sizeof(vamp::BatchCtl)),
                 o_it = take(sizeof(vamp::BatchIter)), o_res = take(ci * 9 * 8);
    if (cudaMalloc(&s->marena, off) != cudaSuccess) return VAMP_ERR_OOM;
    if (cudaMallocHost(&s->hmem, off) != cudaSuccess) return VAMP_ERR_OOM;
    unsigned char* d = (unsigned char*)s->marena;
    unsigned char* h = (unsigned char*)s->hmem;
    s->d_inst = (Params*)(d + o_inst); s->h_inst = (Params*)(h + o_inst);
    s->d_tiles = (int*)(d + o_tiles); s->h_tiles = (int*)(h + o_tiles);
    s->d_comb = (int*)(d + o_comb); s->h_comb = (int*)(h + o_comb);
    s->d_ncalls = (int64_t*)(d + o_nc); s->h_ncalls = (int64_t*)(h + o_nc);
    s->d_iter = (uint32_t*)(d + o_it2); s->h_iter = (uint32_t*)(h + o_it2);
    s->d_pair_off = (int*)(d + o_po); s->h_pair_off = (int*)(h + o_po);
    s->d_pair_prefix = (long long*)(d + o_pp);
    s->d_row_off = (int*)(d + o_ro); s->h_row_off = (int*)(h + o_ro);
    s->d_ctl = (vamp::BatchCtl*)(d + o_ctl);
    s->d_it = (vamp::BatchIter*)(d + o_it); s->h_it = (vamp::BatchIter*)(h + o_it);
    s->d_results = (double*)(d + o_res); s->h_results = (double*)(h + o_res);
    s->mcap_inst = ci;
    s->mcap_pairs = cp;
    return VAMP_OK;
}

// Enqueues one iteration of every request in ints as one multi-instance
// launch on the server stream; tick_finish reads the results once the
// recorded event has completed.
vamp_status tick_launch(vamp_server* s, const std::vector<Req*>& ints)
{
    const int n = (int)ints.size();
    size_t npairs = 0;
    for (Req* r : ints) npairs += r->P.K;
    vamp_status st = grow_multi(s, n, npairs);
    if (st != VAMP_OK) return st;
    size_t smem = 0;
    int max_n = 0;
    s->h_pair_off[0] = 0;
    s->h_row_off[0] = 0;
    for (int i = 0; i < n; ++i) {
        Req* r = ints[i];
        const Params& P = r->P;
        const size_t S = (size_t)(s->fp32 ? P.lay32.bytes : P.lay64.bytes);
        const size_t ds = (size_t)P.d * P.n * 8;
        const size_t fixed = vamp::SMEM_HEAD + vamp::PARAMS_SLOT + ds;
        long t = s->tick_budget > fixed ? (long)((s->tick_budget - fixed) / (2 * S)) : 1;
        t = std::max(1L, std::min(t, (long)P.K));
        smem = std::max(smem, fixed + 2 * (size_t)t * S);
        s->h_inst[i] = P;
        s->h_tiles[i] = (int)t;
        s->h_comb[i] = r->cfg.combine_from;
        s->h_ncalls[i] = r->calls;
        s->h_iter[i] = (uint32_t)r->it_done;
        s->h_pair_off[i + 1] = s->h_pair_off[i] + P.K;
        s->h_row_off[i + 1] = s->h_row_off[i] + P.K * P.d;
        max_n = std::max(max_n, P.n);
    }
    s->h_it->iteration = 0;
    s->h_it->adapt = 3;
    int strat = 0;
    for (Req* r : ints) strat |= r->P.stratified;
    if (smem != s->tick_smem || strat != s->tick_strat) {
        const void* fn = vamp::pass_multi_kernel(s->fp32, s->tick_minb, strat);
        int bps = 0;
        if (vamp::ensure_smem(fn, smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, vamp::PASS_THREADS, smem) != cudaSuccess)
            return VAMP_ERR_CUDA;
        s->tick_smem = smem;
        s->tick_strat = strat;
        s->tick_grid = (bps > 0 ? bps : 1) * s->sm_count;
    }
    cudaStream_t st0 = s->stream;
    cudaError_t e = cudaMemcpyAsync(s->d_inst, s->h_inst, n * sizeof(Params), cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_tiles, s->h_tiles, n * 4, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_comb, s->h_comb, n * 4, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_ncalls, s->h_ncalls, n * 8, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_iter, s->h_iter, n * 4, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_pair_off, s->h_pair_off, (n + 1) * 4, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_row_off, s->h_row_off, (n + 1) * 4, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_it, s->h_it, sizeof(vamp::BatchIter), cudaMemcpyHostToDevice, st0);
    vamp::MultiArgs M{};
    M.inst = s->d_inst;
    M.tiles = s->d_tiles;
    M.combine_from = s->d_comb;
    M.ncalls = s->d_ncalls;
    M.iter = s->d_iter;
    M.pair_off = s->d_pair_off;
    M.pair_prefix = s->d_pair_prefix;
    M.row_off = s->d_row_off;
    M.ctl = s->d_ctl;
    M.it = s->d_it;
    M.results = s->d_results;
    M.n_inst = n;
    M.npairs = (int)npairs;
    M.nrows = s->h_row_off[n];
    M.max_n = max_n;
    M.item_calls = (int64_t)vamp::PASS_THREADS * 8;
    M.any_strat = strat;
    if (e == cudaSuccess) e = vamp::launch_batch_begin(M, st0);
    if (e == cudaSuccess) e = vamp::launch_pass_multi(s->fp32, s->tick_minb, M, s->tick_grid, smem, st0);
    if (e == cudaSuccess) e = vamp::launch_batch_after(M, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_results, s->d_results, (size_t)n * 9 * 8, cudaMemcpyDeviceToHost, st0);
    if (e == cudaSuccess) e = cudaEventRecord(s->tick_ev, st0);
    if (e != cudaSuccess) return VAMP_ERR_CUDA;
    for (Req* r : ints) r->in_tick = true;
    return VAMP_OK;
}

// Results of the launch in flight (its event has completed).
void tick_finish(vamp_server* s, const std::vector<Req*>& ints)
{
    const int n = (int)ints.size();
    for (int i = 0; i < n; ++i) {
        Req* r = ints[i];
        r->in_tick = false;
        const double* x = s->h_results + (size_t)i * 9;
        r->last.integral = x[0];
        r->last.variance = x[1];
        r->last.w_max = x[2];
        r->last.efficiency = x[3];
        r->last.n_calls = (int64_t)x[4];
        r->last.combined = x[5];
        r->last.combined_sigma = x[6];
        r->last.chi2_dof = x[7];
        r->calls_total += (int64_t)x[4];
        s->calls_done += (int64_t)x[4];
        if ((unsigned)x[8]) r->status = ((unsigned)x[8] & vamp::ERR_TIMEOUT) ? VAMP_ERR_TIMEOUT : VAMP_ERR_NUMERIC;
        if (++r->it_done >= r->iterations) {
            r->phase = r->n_events > 0 ? 2 : 3;
            if (r->state_out && r->status == VAMP_OK) {
                // the adapted state, copied on the request's stream before
                // any generation batch (which leaves grids, α and shifts alone)
                const Params& P = r->P;
                const size_t ne = (size_t)P.K * P.d * (P.n + 1);
                cudaError_t e = cudaMemcpyAsync(r->state_out, P.edges64, ne * 8, cudaMemcpyDeviceToDevice, r->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(r->state_out + ne, P.alpha, (size_t)P.K * 8, cudaMemcpyDeviceToDevice, r->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(r->state_out + ne + P.K, P.shift, (size_t)P.K * 8, cudaMemcpyDeviceToDevice,
                                        r->stream);
                if (e == cudaSuccess && r->phase == 3) {
                    // no generation follows: completion waits for the copy
                    e = cudaEventRecord(r->ev, r->stream);
                    if (e == cudaSuccess) r->in_flight = true;
                }
                if (e != cudaSuccess) r->status = VAMP_ERR_CUDA;
            }
        }
    }
    ++s->n_ticks;
}

// Starts the next generation batch of a request on its own stream.
vamp_status gen_launch(vamp_server* s, Req* r)
{
    const Params& P = r->P;
    cudaError_t e = cudaSuccess;
    if (r->gen_b == 0) e = vamp::launch_gen_prepare(P, r->stream);
    if (r->gen_b >= 0x10000u) return VAMP_ERR_LIMIT;
    if (r->max_gen_calls > 0 && (int64_t)r->gen_b * r->gen_batch >= r->max_gen_calls) return VAMP_ERR_LIMIT;
    vamp::PassArgs G{};
    G.tile = r->tile;
    G.ntiles = (P.K + r->tile - 1) / r->tile;
    G.rec_bytes = (int)vamp_record_bytes(P.d);
    G.batch = r->gen_batch;
    G.chunk = r->chunk;
    G.nchunks = r->nchunks;
    G.staging = r->staging;
    G.callidx = r->callidx;
    G.counts = r->counts;
    G.offsets = r->offsets;
    G.field = 0x80000000u | (uint32_t)r->gen_b;  // generation stream 0 of the request
    unsigned char* outp = r->records + r->written * G.rec_bytes;
    if (e == cudaSuccess) e = r->var->launch(P, 1, G, r->grid_gen, r->smem_gen, r->stream);
    if (e == cudaSuccess) e = vamp::launch_gen_finish(P, G, r->n_events - r->written, outp, r->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->h_head, P.sc, offsetof(Scalars, n_hist), cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, r->stream);
    if (e != cudaSuccess) return VAMP_ERR_CUDA;
    r->in_flight = true;
    s->gen_batches += 1;
    return VAMP_OK;
}

void complete(vamp_server* s, Req* r)
{
    r->t_done = clk::now();
    vamp_request_result o{};
    o.id = r->id;
    o.status = r->status;
    o.iterations = r->it_done;
    o.result = r->last;
    o.calls_total = r->calls_total;
    o.events_written = r->written;
    o.events_calls_used = r->used;
    o.events_overweight = r->over;
    o.queue_s = secs(r->t_arrive, r->t_admit);
    o.latency_s = secs(r->t_arrive, r->t_done);
    s->events_done += r->written;
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(o);
    s->n_live -= 1;
}

void scheduler(vamp_server* s)
{
    cudaSetDevice(s->dev);
    bool tick_running = false;
    for (;;) {
        bool progress = false;
        // ---- admission (initialisation enqueued on the request's stream) --
        std::vector<Req*> admitted;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) return;
            if (s->queue.empty() && s->active.empty()) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            // first come, first admitted: stop at the first request that does not fit
            int64_t pending = 0;
            while (!s->queue.empty() && (int)(s->active.size() + admitted.size()) < s->max_slots) {
                Req* r = s->queue.front();
                size_t a0, a, b2, c, dd;
                const int64_t need = (int64_t)request_bytes(r, &a0, &a, &b2, &c, &dd);
                if (s->used_mem + pending + need > s->budget && !(s->active.empty() && admitted.empty())) break;
                s->queue.pop_front();
                admitted.push_back(r);
                pending += need;
            }
        }
        for (Req* r : admitted) {
            progress = true;
            r->status = admit(s, r);
            if (r->status != VAMP_OK) {
                r->t_admit = clk::now();
                complete(s, r);
                free_req(s, r);
                continue;
            }
            s->active.push_back(r);
        }
        // ---- the integration launch in flight ---------------------------
        if (tick_running) {
            const cudaError_t q = cudaEventQuery(s->tick_ev);
            if (q == cudaSuccess) {
                tick_finish(s, s->tick_reqs);
                tick_running = false;
                progress = true;
            } else if (q != cudaErrorNotReady) {
                for (Req* r : s->tick_reqs) { r->in_tick = false; r->status = VAMP_ERR_CUDA; }
                tick_running = false;
            }
        }
        // ---- per request: setup done, generation batches ----------------
        for (Req* r : s->active) {
            if (r->status != VAMP_OK || !r->in_flight) continue;
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) continue;
            r->in_flight = false;
            progress = true;
            if (q != cudaSuccess) { r->status = VAMP_ERR_CUDA; continue; }
            if (r->phase == 0) {
                r->phase = 1;
            } else if (r->phase == 2) {
                r->written += r->h_head->gen_take;
                r->used += r->h_head->gen_used;
                r->over += r->h_head->gen_over;
                if (r->h_head->err) r->status = VAMP_ERR_NUMERIC;
                ++r->gen_b;
                if (r->written >= r->n_events) r->phase = 3;
            }
        }
        // ---- next integration launch: every ready integrating request ----
        if (!tick_running) {
            s->tick_reqs.clear();
            for (Req* r : s->active)
                if (r->phase == 1 && r->status == VAMP_OK && !r->in_flight) s->tick_reqs.push_back(r);
            if (!s->tick_reqs.empty()) {
                const vamp_status st = tick_launch(s, s->tick_reqs);
                if (st != VAMP_OK)
                    for (Req* r : s->tick_reqs) r->status = st;
                else
                    tick_running = true;
                progress = true;
            }
        }
        // ---- generation batches on the requests' streams (overlap) -------
        for (Req* r : s->active)
            if (r->phase == 2 && !r->in_flight && r->status == VAMP_OK) {
                r->status = gen_launch(s, r);
                progress = true;
            }
        // ---- completed requests ------------------------------------------
        std::vector<Req*> keep;
        for (Req* r : s->active) {
            if (r->in_tick || r->in_flight) {
                keep.push_back(r);
                continue;
            }
            if (r->status != VAMP_OK) r->phase = 3;
            if (r->phase == 3) {
                complete(s, r);
                free_req(s, r);
                progress = true;
            } else {
                keep.push_back(r);
            }
        }
        s->active.swap(keep);
        int32_t ni = 0, ng = 0;
        for (Req* r : s->active) (r->phase <= 1 ? ni : ng) += 1;
        s->n_integrating = ni;
        s->n_generating = ng;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->n_queued = (int32_t)s->queue.size();
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" {

vamp_status vamp_server_create(int32_t max_slots, int64_t mem_budget_bytes, int32_t precision, vamp_server** out)
{
    if (!out) return VAMP_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_slots < 1 || mem_budget_bytes < 1 || (precision != VAMP_PREC_FP64 && precision != VAMP_PREC_FP32_EVAL))
        return VAMP_ERR_INVALID_ARG;
    vamp_server* s = new (std::nothrow) vamp_server();
    if (!s) return VAMP_ERR_OOM;
    s->max_slots = max_slots;
    s->budget = mem_budget_bytes;
    s->fp32 = precision == VAMP_PREC_FP32_EVAL;
    if (s->fp32) {
        s->tick_minb = 3;
        s->tick_budget = 72 * 1024;
    }
    if (cudaGetDevice(&s->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return VAMP_ERR_CUDA;
    }
    // the server's own memory pool: freed request memory stays in it (up to
    // the budget) for the next requests
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = s->dev;
    s->head_stride = (offsetof(Scalars, n_hist) + 127) & ~size_t(127);
    s->lanes.resize(max_slots);
    for (int i = max_slots - 1; i >= 0; --i) s->free_lanes.push_back(i);
    if (cudaMemPoolCreate(&s->pool, &pp) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->tick_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&s->h_heads, s->head_stride * (size_t)max_slots) != cudaSuccess) {
        vamp_server_destroy(s);
        return VAMP_ERR_CUDA;
    }
    uint64_t keep = (uint64_t)mem_budget_bytes;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    s->th = std::thread(scheduler, s);
    *out = s;
    return VAMP_OK;
}

vamp_status vamp_server_submit_state(vamp_server* s, const vamp_config* cfg, int32_t iterations, int64_t calls,
                                     int64_t n_events, int64_t max_gen_calls, void* dev_records, double* dev_state,
                                     uint64_t* id_out)
{
    if (!s || !cfg) return VAMP_ERR_INVALID_ARG;
    if (iterations < 1 || calls < 1 || n_events < 0 || max_gen_calls < 0) return VAMP_ERR_INVALID_ARG;
    if (n_events > 0 && (!dev_records || ((uintptr_t)dev_records & 7u))) return VAMP_ERR_INVALID_ARG;
    if ((uintptr_t)dev_state & 7u) return VAMP_ERR_INVALID_ARG;
    Req* r = new (std::nothrow) Req();
    if (!r) return VAMP_ERR_OOM;
    r->cfg = *cfg;
    r->cfg.precision = s->fp32 ? VAMP_PREC_FP32_EVAL : VAMP_PREC_FP64;
    if (cfg->n_channels > 0 && cfg->channels) r->ch.assign(cfg->channels, cfg->channels + cfg->n_channels);
    if (cfg->n_peaks > 0 && cfg->peaks) r->pk.assign(cfg->peaks, cfg->peaks + cfg->n_peaks);
    if (cfg->n_peaks > 0 && cfg->peak_weight) r->w.assign(cfg->peak_weight, cfg->peak_weight + cfg->n_peaks);
    r->cfg.channels = r->ch.data();
    r->cfg.peaks = r->pk.data();
    r->cfg.peak_weight = r->w.data();
    std::string why;
    if (!vamp::build_setup(&r->cfg, r->P, r->S, why)) {
        delete r;
        return VAMP_ERR_INVALID_ARG;
    }
    r->cfg.equiv = nullptr;  // copied into the setup; the caller's table may go away
    r->cfg.n_equiv = 0;
    if (calls > int64_t(0xffffffff) || calls > int64_t(0xffffffff) - (int64_t)r->P.K * r->P.n_min) {
        delete r;
        return VAMP_ERR_INVALID_ARG;
    }
    r->ar = vamp::plan_arena(r->P);
    // generation kernel: the one specialised for this shape if there is one
    const std::vector<const vamp::PassVariant*> cand = vamp::pass_candidates(s->fp32, r->P.d, r->P.n);
    if (cand.empty()) {
        delete r;
        return VAMP_ERR_INVALID_ARG;
    }
    r->var = cand[0];
    r->iterations = iterations;
    r->calls = calls;
    r->n_events = n_events;
    r->max_gen_calls = max_gen_calls;
    r->records = (unsigned char*)dev_records;
    r->state_out = dev_state;
    r->t_arrive = clk::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        s->queue.push_back(r);
        s->n_live += 1;
    }
    s->cv.notify_one();
    if (id_out) *id_out = r->id;
    return VAMP_OK;
}

vamp_status vamp_server_submit(vamp_server* s, const vamp_config* cfg, int32_t iterations, int64_t calls,
                               int64_t n_events, int64_t max_gen_calls, void* dev_records, uint64_t* id_out)
{
    return vamp_server_submit_state(s, cfg, iterations, calls, n_events, max_gen_calls, dev_records, nullptr,
                                    id_out);
}

int32_t vamp_server_poll(vamp_server* s, vamp_request_result* out, int32_t max_results)
{
    if (!s || !out || max_results < 1) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    const int32_t k = (int32_t)std::min<size_t>(s->done.size(), (size_t)max_results);
    for (int32_t i = 0; i < k; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + k);
    return k;
}

vamp_status vamp_server_wait_idle(vamp_server* s, double timeout_s)
{
    if (!s) return VAMP_ERR_INVALID_ARG;
    const clk::time_point t0 = clk::now();
    for (;;) {
        if (s->n_live.load() == 0) return VAMP_OK;
        if (secs(t0, clk::now()) > timeout_s) return VAMP_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
}

vamp_status vamp_server_stats(const vamp_server* s, int64_t* ticks, int64_t* calls, int64_t* events,
                              int64_t* mem_in_use)
{
    if (!s) return VAMP_ERR_INVALID_ARG;
    if (ticks) *ticks = s->n_ticks;
    if (calls) *calls = s->calls_done;
    if (events) *events = s->events_done;
    if (mem_in_use) *mem_in_use = s->used_mem;
    return VAMP_OK;
}

vamp_status vamp_server_load(const vamp_server* s, int32_t* queued, int32_t* integrating, int32_t* generating,
                             int64_t* gen_batches)
{
    if (!s) return VAMP_ERR_INVALID_ARG;
    if (queued) *queued = s->n_queued;
    if (integrating) *integrating = s->n_integrating;
    if (generating) *generating = s->n_generating;
    if (gen_batches) *gen_batches = s->gen_batches;
    return VAMP_OK;
}

void vamp_server_destroy(vamp_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Req* r : s->queue) delete r;
        s->queue.clear();
    }
    s->cv.notify_one();
    if (s->th.joinable()) s->th.join();
    if (s->stream) cudaStreamSynchronize(s->stream);  // a launch still in flight
    for (Req* r : s->active) free_req(s, r);
    cudaDeviceSynchronize();  // frees and work of the lanes' streams
    for (vamp_server::Lane& l : s->lanes) {
        if (l.ev) cudaEventDestroy(l.ev);
        if (l.stream) cudaStreamDestroy(l.stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->tick_ev) cudaEventDestroy(s->tick_ev);
    cudaFreeHost(s->h_heads);
    cudaFree(s->marena);
    cudaFreeHost(s->hmem);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"

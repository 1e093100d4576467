// vamp_api.cu -- the C ABI of include/vamp.h: validation, device state,
// launch order, result read-back.  Every step of the integration runs in the
// kernels of vamp_kernels.cu; this file only marshals.
#include "../../include/vamp.h"
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using vamp::MapRec;
using vamp::Params;
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
    int grid_pass = 0;         // persistent grid of the integration pass kernel
    int grid_gen = 0;          // CTAs per SM x SMs for generation
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

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool check_maps(const vamp_map_desc* m, int cnt, int d, std::string& why)
{
    for (int q = 0; q < cnt; ++q) {
        const vamp_map_desc& r = m[q];
        if (r.n_mapped < 0 || r.n_mapped > vamp::MAXMAP) { why = "n_mapped out of range"; return false; }
        unsigned seen = 0;
        for (int s = 0; s < r.n_mapped; ++s) {
            const int k = r.coord[s];
            if (k < 0 || k >= d) { why = "mapped coordinate out of range"; return false; }
            if (seen & (1u << k)) { why = "coordinate mapped twice"; return false; }
            seen |= 1u << k;
            if (r.kind[s] == VAMP_MAP_BW) {
                if (!(r.b[s] > 0.0) || !std::isfinite(r.a[s]) || !std::isfinite(r.b[s])) {
                    why = "Breit-Wigner width must be > 0";
                    return false;
                }
            } else if (r.kind[s] == VAMP_MAP_POW) {
                if (!(r.b[s] >= 0.0) || !std::isfinite(r.b[s])) { why = "power-law delta must be >= 0"; return false; }
            } else if (r.kind[s] != VAMP_MAP_ID) {
                why = "unknown map kind";
                return false;
            }
        }
    }
    return true;
}

template <typename T>
MapRec<T> make_rec(const vamp_map_desc& r, double weight, double zinv, int d)
{
    MapRec<T> o;
    std::memset(&o, 0, sizeof o);
    o.nmap = r.n_mapped;
    // peak weight times Z^-(d - n_mapped): the Gaussian normalisation of the
    // coordinates the peak does not map
    o.wz = (T)(weight * std::pow(zinv, (double)(d - r.n_mapped)));
    for (int s = 0; s < r.n_mapped; ++s) {
        const int k = r.coord[s];
        o.mask |= 1u << k;
        o.slotpack |= (uint64_t)s << (4 * k);
        o.kind[s] = r.kind[s];
        if (r.kind[s] == VAMP_MAP_BW) {
            const double m = r.a[s], G = r.b[s];
            const double A = std::atan((1.0 - m) / G) + std::atan(m / G); // ∫_0^1 Γ/((p-m)²+Γ²)
            o.m[s] = (T)m;
            o.G[s] = (T)G;
            o.invG[s] = (T)(1.0 / G);
            o.A[s] = (T)A;
            o.GinvA[s] = (T)(G / A);
            o.invA[s] = (T)(1.0 / A);
            o.t0[s] = (T)std::atan(m / G);
        } else if (r.kind[s] == VAMP_MAP_POW) {
            const double del = r.b[s];
            o.del[s] = (T)del;
            // 1 / ∫_0^1 (p+δ)^-0.8 dp
            o.invPowN[s] = (T)(1.0 / (5.0 * (std::pow(1.0 + del, 0.2) - std::pow(del, 0.2))));
        }
    }
    return o;
}

bool same_maps(const vamp_map_desc& a, const vamp_map_desc& b)
{
    if (a.n_mapped != b.n_mapped) return false;
    for (int s = 0; s < a.n_mapped; ++s)
        if (a.coord[s] != b.coord[s] || a.kind[s] != b.kind[s] || a.a[s] != b.a[s] || a.b[s] != b.b[s])
            return false;
    return true;
}

// Lookup-block layout for elements of `esz` bytes (see vamp_device.cuh).
vamp::BlkLayout make_layout(int d, int n, int esz)
{
    vamp::BlkLayout L{};
    const int per16 = 16 / esz;
    L.Es = (n + 1 + per16 - 1) / per16 * per16;
    L.Dn = (n + per16 - 1) / per16 * per16;
    int lshift = 0;
    while ((1 << lshift) < n) ++lshift;
    lshift += 1;                      // two cells per bin on a uniform grid
    if (lshift < 2) lshift = 2;
    L.lshift = lshift;
    L.Ts = ((1 << lshift) + 1 + 15) / 16 * 16;
    L.off_dens = d * L.Es * esz;
    L.off_tab = L.off_dens + d * L.Dn * esz;
    L.off_span = L.off_tab + d * L.Ts;
    L.bytes = (L.off_span + d + 15) / 16 * 16;
    return L;
}

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
    }
    return "VAMP_ERR_UNKNOWN";
}

const char* vamp_last_error(const vamp_ctx* c) { return c ? c->err.c_str() : ""; }

int64_t vamp_record_bytes(int32_t d) { return ((4 * (int64_t)d + 7) & ~int64_t(7)) + 8; }

void vamp_destroy(vamp_ctx* c)
{
    if (!c) return;
    {
        DeviceGuard g(c->dev);
        if (c->stream) cudaStreamSynchronize(c->stream);
        cudaFree(c->arena);
        cudaFree(c->g_staging);
        cudaFree(c->g_callidx);
        cudaFree(c->g_counts);
        cudaFree(c->g_offsets);
        cudaFreeHost(c->h_head);
        if (c->ev[0]) cudaEventDestroy(c->ev[0]);
        if (c->ev[1]) cudaEventDestroy(c->ev[1]);
    }
    delete c;
}

vamp_status vamp_create(const vamp_config* cfg, void* cuda_stream, vamp_ctx** out)
{
    if (!out) return VAMP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg) return VAMP_ERR_INVALID_ARG;
    const int d = cfg->d, K = cfg->n_channels, n = cfg->n_bins, P = cfg->n_peaks;
    if (d < 1 || d > vamp::DMAX || K < 1 || n < 1 || n > vamp::MAX_BINS || P < 1 || !cfg->channels ||
        !cfg->peaks || !cfg->peak_weight)
        return VAMP_ERR_INVALID_ARG;
    std::string why;
    if (!check_maps(cfg->channels, K, d, why) || !check_maps(cfg->peaks, P, d, why)) return VAMP_ERR_INVALID_ARG;
    if (!(cfg->gauss_sigma >= 0.0) || !(cfg->grid_alpha > 0.0) || !std::isfinite(cfg->beta) || cfg->n_min < 1 ||
        cfg->gen_batch < 0 || cfg->gen_batch > (int64_t(1) << 24) ||
        (cfg->precision != VAMP_PREC_FP64 && cfg->precision != VAMP_PREC_FP32_EVAL))
        return VAMP_ERR_INVALID_ARG;
    for (int q = 0; q < P; ++q)
        if (!std::isfinite(cfg->peak_weight[q])) return VAMP_ERR_INVALID_ARG;

    vamp_ctx* c = new (std::nothrow) vamp_ctx();
    if (!c) return VAMP_ERR_OOM;
    if (cudaGetDevice(&c->dev) != cudaSuccess) { delete c; return VAMP_ERR_CUDA; }
    c->stream = (cudaStream_t)cuda_stream;
    c->d = d; c->K = K; c->n = n; c->P = P;
    c->fp32 = cfg->precision == VAMP_PREC_FP32_EVAL;
    c->combine_from = cfg->combine_from;
    c->gen_batch = cfg->gen_batch > 0 ? cfg->gen_batch : (int64_t(1) << 20);

    Params& pr = c->prm;
    pr.d = d; pr.K = K; pr.n = n; pr.P = P;
    pr.key0 = (uint32_t)(cfg->seed & 0xffffffffu);
    pr.key1 = (uint32_t)(cfg->seed >> 32);
    pr.request = cfg->request_id;
    pr.n_min = cfg->n_min;
    pr.grid_alpha = cfg->grid_alpha;
    pr.beta = cfg->beta;
    pr.smooth = cfg->smooth;
    pr.omega_mode = cfg->omega_mode;
    // Gaussian factor exp(-(p-c)^2 / (2σ^2)) / Z as 2^-(p-c)^2 gk2 (gk2 = log2(e)/(2σ^2));
    // σ = 0 switches it off (factor 1)
    double zinv = 1.0;
    if (cfg->gauss_sigma > 0.0) {
        const double s = cfg->gauss_sigma, cc = cfg->gauss_centre;
        double Z;
        if (cfg->gauss_norm == VAMP_GAUSS_NORM_REAL_LINE) Z = s * std::sqrt(2.0 * M_PI);
        else Z = s * std::sqrt(M_PI / 2.0) * (std::erf((1.0 - cc) / (s * M_SQRT2)) + std::erf(cc / (s * M_SQRT2)));
        zinv = 1.0 / Z;
        pr.gcen = cc;
        pr.gk2 = M_LOG2E / (2.0 * s * s);
        pr.gcen_f = (float)cc;
        pr.gk2_f = (float)pr.gk2;
    }
    pr.matching = P == K;
    for (int q = 0; pr.matching && q < K; ++q)
        if (!same_maps(cfg->channels[q], cfg->peaks[q])) pr.matching = 0;
    pr.lay64 = make_layout(d, n, 8);
    pr.lay32 = make_layout(d, n, 4);

    // one arena for all device state
    const size_t rows = (size_t)K * d;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += align256(bytes); return o; };
    const size_t o_e64 = take(rows * (n + 1) * 8);
    const size_t o_lk64 = take((size_t)K * pr.lay64.bytes), o_lk32 = take((size_t)K * pr.lay32.bytes);
    const size_t o_al = take(K * 8), o_al32 = take(K * 4), o_sh = take(K * 8), o_ac = take(K * 8);
    const size_t o_nc = take(K * 8), o_pc = take((K + 1) * 8), o_D = take(rows * n * 8);
    const size_t o_cs = take(2 * K * 8), o_ic = take(K * 8), o_vc = take(K * 8), o_wc = take(K * 8);
    const size_t o_ch64 = take(K * sizeof(MapRec<double>)), o_ch32 = take(K * sizeof(MapRec<float>));
    const size_t o_pk64 = take(P * sizeof(MapRec<double>)), o_pk32 = take(P * sizeof(MapRec<float>));
    const size_t o_sc = take(sizeof(Scalars));
    DeviceGuard g(c->dev);
    cudaError_t e = cudaMalloc(&c->arena, off);
    if (e != cudaSuccess) { delete c; return e == cudaErrorMemoryAllocation ? VAMP_ERR_OOM : VAMP_ERR_CUDA; }
    e = cudaMallocHost((void**)&c->h_head, sizeof(Scalars));
    if (e != cudaSuccess) { vamp_destroy(c); return VAMP_ERR_OOM; }
    char* b = (char*)c->arena;
    pr.edges64 = (double*)(b + o_e64);
    pr.lk64 = (unsigned char*)(b + o_lk64); pr.lk32 = (unsigned char*)(b + o_lk32);
    pr.alpha = (double*)(b + o_al); pr.alpha32 = (float*)(b + o_al32);
    pr.shift = (double*)(b + o_sh); pr.Acum = (double*)(b + o_ac);
    pr.Nc = (int64_t*)(b + o_nc); pr.Pc = (int64_t*)(b + o_pc); pr.D = (double*)(b + o_D);
    pr.csum = (double*)(b + o_cs); pr.Ic = (double*)(b + o_ic); pr.Vc = (double*)(b + o_vc);
    pr.Wc = (double*)(b + o_wc);
    pr.ch64 = (MapRec<double>*)(b + o_ch64); pr.ch32 = (MapRec<float>*)(b + o_ch32);
    pr.pk64 = (MapRec<double>*)(b + o_pk64); pr.pk32 = (MapRec<float>*)(b + o_pk32);
    pr.sc = (Scalars*)(b + o_sc);

    // host images: uniform grids ξ_j = j/n, α_c = 1/K (§3.4, §3.5)
    std::vector<double> edges(rows * (n + 1)), alpha(K, 1.0 / (double)K);
    for (size_t r = 0; r < rows; ++r)
        for (int j = 0; j <= n; ++j) edges[r * (n + 1) + j] = (double)j / (double)n;
    std::vector<MapRec<double>> ch64(K), pk64(P);
    std::vector<MapRec<float>> ch32(K), pk32(P);
    for (int q = 0; q < K; ++q) {
        // with matching peaks the channel record carries the peak weight too
        const double w = pr.matching ? cfg->peak_weight[q] : 0.0;
        ch64[q] = make_rec<double>(cfg->channels[q], w, zinv, d);
        ch32[q] = make_rec<float>(cfg->channels[q], w, zinv, d);
    }
    for (int q = 0; q < P; ++q) {
        pk64[q] = make_rec<double>(cfg->peaks[q], cfg->peak_weight[q], zinv, d);
        pk32[q] = make_rec<float>(cfg->peaks[q], cfg->peak_weight[q], zinv, d);
    }
    vamp_status st = VAMP_OK;
#define CREATE_CK(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) { st = cuda_fail(c, e_, #call); goto create_fail; }        \
    } while (0)
    CREATE_CK(cudaMemsetAsync(c->arena, 0, off, c->stream));
    CREATE_CK(cudaMemcpyAsync(pr.edges64, edges.data(), edges.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(cudaMemcpyAsync(pr.alpha, alpha.data(), K * 8, cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(cudaMemcpyAsync((void*)pr.ch64, ch64.data(), K * sizeof(MapRec<double>), cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(cudaMemcpyAsync((void*)pr.ch32, ch32.data(), K * sizeof(MapRec<float>), cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(cudaMemcpyAsync((void*)pr.pk64, pk64.data(), P * sizeof(MapRec<double>), cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(cudaMemcpyAsync((void*)pr.pk32, pk32.data(), P * sizeof(MapRec<float>), cudaMemcpyHostToDevice, c->stream));
    CREATE_CK(vamp::launch_derive(pr, c->stream));
    {
        // channels per staged tile: two tile buffers plus the d-value
        // accumulators within ~112 KB, so that two CTAs share an SM
        const int S = c->fp32 ? pr.lay32.bytes : pr.lay64.bytes;
        const size_t ds = (size_t)d * n * 8;
        const size_t budget = 112 * 1024;
        int tile = (int)((budget - vamp::SMEM_HEAD - ds) / (2 * (size_t)S));
        if (tile < 1) tile = 1;
        if (tile > K) tile = K;
        c->tile = tile;
        c->smem_pass = vamp::SMEM_HEAD + 2 * (size_t)tile * S + ds;
        c->smem_gen = vamp::SMEM_HEAD + 2 * (size_t)tile * S;
        int maxsm = 0;
        CREATE_CK(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
        if ((int)c->smem_pass > maxsm) { st = fail(c, VAMP_ERR_INVALID_ARG, "grid too large for shared memory"); goto create_fail; }
        // the limit is per kernel, not per context: only ever raise it, so
        // that contexts created earlier keep theirs
        for (int mode = 0; mode < 2; ++mode) {
            const size_t need = mode ? c->smem_gen : c->smem_pass;
            cudaFuncAttributes fa{};
            CREATE_CK(cudaFuncGetAttributes(&fa, vamp::pass_kernel(c->fp32, mode)));
            if (fa.maxDynamicSharedSizeBytes < (int)need)
                CREATE_CK(cudaFuncSetAttribute(vamp::pass_kernel(c->fp32, mode),
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
        }
        int b0 = 0, b1 = 0;
        CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, vamp::pass_kernel(c->fp32, 0),
                                                                vamp::PASS_THREADS, c->smem_pass));
        CREATE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, vamp::pass_kernel(c->fp32, 1),
                                                                vamp::PASS_THREADS, c->smem_gen));
        CREATE_CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev));
        c->grid_pass = (b0 > 0 ? b0 : 1) * c->sm_count;
        c->grid_gen = (b1 > 0 ? b1 : 1) * c->sm_count;
    }
    CREATE_CK(cudaStreamSynchronize(c->stream));
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
    if (n_calls + (int64_t)c->K * c->prm.n_min > int64_t(0xffffffff))
        return fail(c, VAMP_ERR_INVALID_ARG, "too many calls for a 32-bit call counter");
    DeviceGuard g(c->dev);
    VAMP_CK(c, vamp::launch_begin_pass(c->prm, n_calls, c->stream));
    vamp_status s = read_head(c);
    if (s != VAMP_OK) return s;
    if (n_total) *n_total = c->h_head->n_total;
    return VAMP_OK;
}

vamp_status vamp_sample_pass(vamp_ctx* c, int64_t n_calls, uint32_t iteration, vamp_pass_result* out)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!out) return fail(c, VAMP_ERR_INVALID_ARG, "out is required");
    if (n_calls < 1) return fail(c, VAMP_ERR_INVALID_ARG, "n_calls must be >= 1");
    if (iteration >= 0x80000000u) return fail(c, VAMP_ERR_INVALID_ARG, "iteration must be < 2^31");
    if (n_calls + (int64_t)c->K * c->prm.n_min > int64_t(0xffffffff))
        return fail(c, VAMP_ERR_INVALID_ARG, "too many calls for a 32-bit call counter");
    DeviceGuard g(c->dev);
    const Params& P = c->prm;
    VAMP_CK(c, cudaMemsetAsync(P.D, 0, (size_t)c->K * c->d * c->n * 8, c->stream));
    VAMP_CK(c, cudaMemsetAsync(P.csum, 0, (size_t)2 * c->K * 8, c->stream));
    VAMP_CK(c, vamp::launch_begin_pass(P, n_calls, c->stream));
    if (c->prof) VAMP_CK(c, cudaEventRecord(c->ev[0], c->stream));
    vamp::PassArgs A{};
    A.field = iteration;
    A.tile = c->tile;
    A.ntiles = (c->K + c->tile - 1) / c->tile;
    VAMP_CK(c, vamp::launch_pass(P, c->fp32, 0, A, c->grid_pass, c->smem_pass, c->stream));
    if (c->prof) VAMP_CK(c, cudaEventRecord(c->ev[1], c->stream));
    VAMP_CK(c, vamp::launch_finish_pass(P, (int)iteration >= c->combine_from ? 1 : 0, c->stream));
    vamp_status s = read_head(c);
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

vamp_status vamp_refine_grids(vamp_ctx* c)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (!c->have_pass) return fail(c, VAMP_ERR_STATE, "refine before any sampling pass");
    DeviceGuard g(c->dev);
    VAMP_CK(c, vamp::launch_refine(c->prm, c->stream));
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
    const int64_t chunk = (int64_t)vamp::PASS_THREADS * (c->fp32 ? vamp::CPT32 : vamp::CPT64);
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
    vamp::PassArgs G{};
    G.tile = c->tile;
    G.ntiles = (c->K + c->tile - 1) / c->tile;
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
        VAMP_CK(c, vamp::launch_pass(c->prm, c->fp32, 1, G, grid, c->smem_gen, c->stream));
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
    VAMP_CK(c, cudaStreamSynchronize(c->stream));
    c->have_pass = 1;
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
    char* q = (char*)buf;
    vamp::EvalArgs A{};
    A.mode = mode; A.field = field; A.call0 = call0; A.count = count;
    A.x = (double*)q; q += align256(nx * 8);
    A.p = (double*)q; q += align256(nx * 8);
    A.jf = (int*)q; q += align256(nx * 4);
    A.fgwc = (double*)q; q += align256((size_t)count * 32);
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
    return VAMP_OK;
}

vamp_status vamp_kernel_stats(vamp_ctx* c, double* sample_ms, int64_t* sample_launches, double* gen_ms,
                              int64_t* gen_launches)
{
    if (!c) return VAMP_ERR_INVALID_ARG;
    if (sample_ms) *sample_ms = c->prof_sample_ms;
    if (sample_launches) *sample_launches = c->prof_sample_n;
    if (gen_ms) *gen_ms = c->prof_gen_ms;
    if (gen_launches) *gen_launches = c->prof_gen_n;
    return VAMP_OK;
}

}  // extern "C"

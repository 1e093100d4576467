// vamp_noalloc.cu -- vamp_sample_pass_static: one sampling pass without any
// device or host allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: code that runs inside a
// framework which owns every byte of device memory through its own pool
// (a serving engine with a fixed memory plan, a caller that measured its
// footprint up front), or code on a path where a device allocation could
// block or fail at an unpredictable moment.  This entry point serves them:
// the caller passes the grid state and the output buffers, and every
// working array of the pass (lookup blocks, map records, call allocation,
// accumulators, scalars) lives in one statically sized device array that
// the library's image carries.  Every GPU that loads the library holds that
// array (VAMP_STATIC_SCRATCH_BYTES) until the process exits.
//
// The array is shared by all calls: each call clears the parts that must
// start at zero, and calls that overlap on the GPU (two streams, two host
// threads) race on it.  The device address of the array is looked up once
// per device, by the first call made with that device current; make that
// first call before any stream capture.
#include "../../include/vamp.h"
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

using vamp::MapRec;
using vamp::Params;
using vamp::Scalars;

namespace {

constexpr size_t VAMP_STATIC_SCRATCH_BYTES = size_t(8) << 20;  // 8 MiB
constexpr int MAX_DEVICES = 128;

__device__ __align__(256) unsigned char g_scratch[VAMP_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

void put_msg(char* buf, int32_t len, const char* msg)
{
    if (buf && len > 0) {
        std::snprintf(buf, (size_t)len, "%s", msg);
    }
}

bool maps_ok(const vamp_map_desc* m, int cnt, int d)
{
    for (int q = 0; q < cnt; ++q) {
        const vamp_map_desc& r = m[q];
        if (r.n_mapped < 0 || r.n_mapped > vamp::MAXMAP) return false;
        unsigned seen = 0;
        for (int s = 0; s < r.n_mapped; ++s) {
            const int k = r.coord[s];
            if (k < 0 || k >= d || (seen & (1u << k))) return false;
            seen |= 1u << k;
            if (r.kind[s] == VAMP_MAP_BW) {
                if (!(r.b[s] > 0.0) || !std::isfinite(r.a[s]) || !std::isfinite(r.b[s])) return false;
            } else if (r.kind[s] == VAMP_MAP_POW) {
                if (!(r.b[s] >= 0.0) || !std::isfinite(r.b[s])) return false;
            } else if (r.kind[s] != VAMP_MAP_ID) {
                return false;
            }
        }
    }
    return true;
}

template <typename T>
MapRec<T> rec_of(const vamp_map_desc& r, double weight, double zinv, int d)
{
    MapRec<T> o;
    std::memset(&o, 0, sizeof o);
    o.nmap = r.n_mapped;
    o.wz = (T)(weight * std::pow(zinv, (double)(d - r.n_mapped)));
    for (int s = 0; s < r.n_mapped; ++s) {
        const int k = r.coord[s];
        o.mask |= 1u << k;
        o.slotpack |= (uint64_t)s << (4 * k);
        o.kind[s] = r.kind[s];
        if (r.kind[s] == VAMP_MAP_BW) {
            const double m = r.a[s], G = r.b[s];
            const double A = std::atan((1.0 - m) / G) + std::atan(m / G);
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
            o.invPowN[s] = (T)(1.0 / (5.0 * (std::pow(1.0 + del, 0.2) - std::pow(del, 0.2))));
        }
    }
    return o;
}

bool same(const vamp_map_desc& a, const vamp_map_desc& b)
{
    if (a.n_mapped != b.n_mapped) return false;
    for (int s = 0; s < a.n_mapped; ++s)
        if (a.coord[s] != b.coord[s] || a.kind[s] != b.kind[s] || a.a[s] != b.a[s] || a.b[s] != b.b[s])
            return false;
    return true;
}

vamp::BlkLayout layout_of(int d, int n, int esz)
{
    vamp::BlkLayout L{};
    const int per16 = 16 / esz;
    L.Es = (n + 1 + per16 - 1) / per16 * per16;
    L.Dn = (n + per16 - 1) / per16 * per16;
    int lshift = 0;
    while ((1 << lshift) < n) ++lshift;
    lshift += 1;
    if (lshift < 2) lshift = 2;
    L.lshift = lshift;
    L.Ts = ((1 << lshift) + 1 + 15) / 16 * 16;
    L.off_dens = d * L.Es * esz;
    L.off_tab = L.off_dens + d * L.Dn * esz;
    L.off_span = L.off_tab + d * L.Ts;
    L.bytes = (L.off_span + d + 15) / 16 * 16;
    return L;
}

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_ptr(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" vamp_status vamp_sample_pass_static(const vamp_config* cfg, const double* dev_edges,
                                               const double* dev_alpha, const double* dev_shift,
                                               int64_t n_calls, uint32_t iteration, void* cuda_stream,
                                               double* dev_D_out, vamp_pass_result* out, char* err_msg,
                                               int32_t err_len)
{
    put_msg(err_msg, err_len, "");
    if (!cfg || !dev_edges || !dev_alpha || !dev_shift || !out) {
        put_msg(err_msg, err_len, "cfg, dev_edges, dev_alpha, dev_shift and out are required");
        return VAMP_ERR_INVALID_ARG;
    }
    const int d = cfg->d, K = cfg->n_channels, n = cfg->n_bins, P = cfg->n_peaks;
    if (d < 1 || d > vamp::DMAX || K < 1 || n < 1 || n > vamp::MAX_BINS || P < 1 || !cfg->channels ||
        !cfg->peaks || !cfg->peak_weight || !maps_ok(cfg->channels, K, d) || !maps_ok(cfg->peaks, P, d) ||
        !(cfg->gauss_sigma >= 0.0) || cfg->n_min < 1 ||
        (cfg->precision != VAMP_PREC_FP64 && cfg->precision != VAMP_PREC_FP32_EVAL)) {
        put_msg(err_msg, err_len, "invalid problem description");
        return VAMP_ERR_INVALID_ARG;
    }
    if (n_calls < 1 || iteration >= 0x80000000u || n_calls + (int64_t)K * cfg->n_min > int64_t(0xffffffff)) {
        put_msg(err_msg, err_len, "n_calls must be >= 1, iteration < 2^31, total calls < 2^32");
        return VAMP_ERR_INVALID_ARG;
    }
    const int fp32 = cfg->precision == VAMP_PREC_FP32_EVAL;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    Params pr{};
    pr.d = d; pr.K = K; pr.n = n; pr.P = P;
    pr.key0 = (uint32_t)(cfg->seed & 0xffffffffu);
    pr.key1 = (uint32_t)(cfg->seed >> 32);
    pr.request = cfg->request_id;
    pr.n_min = cfg->n_min;
    pr.grid_alpha = cfg->grid_alpha;
    pr.beta = cfg->beta;
    pr.smooth = cfg->smooth;
    pr.omega_mode = cfg->omega_mode;
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
        if (!same(cfg->channels[q], cfg->peaks[q])) pr.matching = 0;
    pr.lay64 = layout_of(d, n, 8);
    pr.lay32 = layout_of(d, n, 4);

    // carve the static array
    const size_t rows = (size_t)K * d;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += a256(bytes); return o; };
    const size_t o_lk64 = take((size_t)K * pr.lay64.bytes), o_lk32 = take((size_t)K * pr.lay32.bytes);
    const size_t o_al32 = take(K * 4), o_sh = take(K * 8), o_ac = take(K * 8);
    const size_t o_nc = take(K * 8), o_pc = take((K + 1) * 8), o_D = take(rows * n * 8);
    const size_t o_cs = take(2 * K * 8), o_ic = take(K * 8), o_vc = take(K * 8), o_wc = take(K * 8);
    const size_t o_ch64 = take(K * sizeof(MapRec<double>)), o_ch32 = take(K * sizeof(MapRec<float>));
    const size_t o_pk64 = take(P * sizeof(MapRec<double>)), o_pk32 = take(P * sizeof(MapRec<float>));
    const size_t o_sc = take(sizeof(Scalars));
    if (off > VAMP_STATIC_SCRATCH_BYTES) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "problem needs %zu bytes of scratch; the static limit is %zu bytes", off,
                      VAMP_STATIC_SCRATCH_BYTES);
        put_msg(err_msg, err_len, msg);
        return VAMP_ERR_INVALID_ARG;
    }
    // shared memory of the pass kernel: same tile rule as vamp_create
    const int S = fp32 ? pr.lay32.bytes : pr.lay64.bytes;
    const size_t ds = (size_t)d * n * 8;
    int tile = (int)((112 * 1024 - vamp::SMEM_HEAD - ds) / (2 * (size_t)S));
    if (tile < 1) tile = 1;
    if (tile > K) tile = K;
    const size_t smem = vamp::SMEM_HEAD + 2 * (size_t)tile * S + ds;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    unsigned char* base = nullptr;
    if (e == cudaSuccess) e = scratch_ptr(dev, &base);
    int maxsm = 0, sms = 0, bps = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && (int)smem > maxsm) {
        put_msg(err_msg, err_len, "grid too large for shared memory");
        return VAMP_ERR_INVALID_ARG;
    }
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        // raise (never lower) the kernel's dynamic shared-memory limit, which
        // contexts created with vamp_create may also rely on
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, vamp::pass_kernel(fp32, 0));
        if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < (int)smem)
            e = cudaFuncSetAttribute(vamp::pass_kernel(fp32, 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
    }
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, vamp::pass_kernel(fp32, 0), vamp::PASS_THREADS, smem);
    if (e != cudaSuccess) {
        put_msg(err_msg, err_len, cudaGetErrorString(e));
        return VAMP_ERR_CUDA;
    }
    pr.lk64 = base + o_lk64;
    pr.lk32 = base + o_lk32;
    pr.edges64 = const_cast<double*>(dev_edges);  // read only by the kernels launched here
    pr.alpha = const_cast<double*>(dev_alpha);    // read only by the kernels launched here
    pr.alpha32 = (float*)(base + o_al32);
    pr.shift = (double*)(base + o_sh);
    pr.Acum = (double*)(base + o_ac);
    pr.Nc = (int64_t*)(base + o_nc);
    pr.Pc = (int64_t*)(base + o_pc);
    pr.D = (double*)(base + o_D);
    pr.csum = (double*)(base + o_cs);
    pr.Ic = (double*)(base + o_ic);
    pr.Vc = (double*)(base + o_vc);
    pr.Wc = (double*)(base + o_wc);
    pr.ch64 = (MapRec<double>*)(base + o_ch64);
    pr.ch32 = (MapRec<float>*)(base + o_ch32);
    pr.pk64 = (MapRec<double>*)(base + o_pk64);
    pr.pk32 = (MapRec<float>*)(base + o_pk32);
    pr.sc = (Scalars*)(base + o_sc);

    std::vector<MapRec<double>> ch64(K), pk64(P);
    std::vector<MapRec<float>> ch32(K), pk32(P);
    for (int q = 0; q < K; ++q) {
        const double w = pr.matching ? cfg->peak_weight[q] : 0.0;
        ch64[q] = rec_of<double>(cfg->channels[q], w, zinv, d);
        ch32[q] = rec_of<float>(cfg->channels[q], w, zinv, d);
    }
    for (int q = 0; q < P; ++q) {
        pk64[q] = rec_of<double>(cfg->peaks[q], cfg->peak_weight[q], zinv, d);
        pk32[q] = rec_of<float>(cfg->peaks[q], cfg->peak_weight[q], zinv, d);
    }
    // everything that must start from zero: accumulators and scalars
    e = cudaMemsetAsync(base + o_D, 0, rows * n * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_cs, 0, 2 * K * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_sc, 0, sizeof(Scalars), stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pr.shift, dev_shift, K * 8, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)pr.ch64, ch64.data(), K * sizeof(MapRec<double>), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)pr.ch32, ch32.data(), K * sizeof(MapRec<float>), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)pr.pk64, pk64.data(), P * sizeof(MapRec<double>), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)pr.pk32, pk32.data(), P * sizeof(MapRec<float>), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = vamp::launch_derive(pr, stream);
    if (e == cudaSuccess) e = vamp::launch_begin_pass(pr, n_calls, stream);
    if (e == cudaSuccess) {
        vamp::PassArgs A{};
        A.field = iteration;
        A.tile = tile;
        A.ntiles = (K + tile - 1) / tile;
        e = vamp::launch_pass(pr, fp32, 0, A, (bps > 0 ? bps : 1) * sms, smem, stream);
    }
    if (e == cudaSuccess) e = vamp::launch_finish_pass(pr, 0, stream);
    if (e == cudaSuccess && dev_D_out)
        e = cudaMemcpyAsync(dev_D_out, pr.D, rows * n * 8, cudaMemcpyDeviceToDevice, stream);
    Scalars head;  // only the head fields are copied back
    const size_t head_bytes = offsetof(Scalars, n_hist);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&head, pr.sc, head_bytes, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        put_msg(err_msg, err_len, cudaGetErrorString(e));
        return VAMP_ERR_CUDA;
    }
    out->integral = head.res[0];
    out->variance = head.res[1];
    out->w_max = head.res[2];
    out->efficiency = head.res[3];
    out->n_calls = head.n_total;
    out->combined = 0.0;
    out->combined_sigma = 0.0;
    out->chi2_dof = 0.0;
    if (head.err & vamp::ERR_TIMEOUT) {
        put_msg(err_msg, err_len, "a bounded wait for staged grid data gave up; results are incomplete");
        return VAMP_ERR_TIMEOUT;
    }
    if (head.err & vamp::ERR_NONFINITE) {
        put_msg(err_msg, err_len, "a non-finite weight was produced (counted as w = 0)");
        return VAMP_ERR_NUMERIC;
    }
    return VAMP_OK;
}

// vamp_noalloc.cu -- vamp_sample_pass_static: one sampling pass that makes
// no device-memory allocation.
//
// Some callers cannot let a library call cudaMalloc: code that runs inside a
// framework which owns every byte of device memory through its own pool
// (a serving engine with a fixed memory plan, a caller that measured its
// footprint up front), or code on a path where a device allocation could
// block or fail at an unpredictable moment.  This entry point serves them:
// the caller passes the grid state and the output buffers, and every
// working array of the pass (lookup blocks, map records, call allocation,
// accumulators, scalars) lives in one statically sized device array that
// the library's image carries.  Every GPU that loads the library's device
// code holds that array (VAMP_STATIC_SCRATCH_BYTES) until the process exits.
// With CUDA's default lazy module loading the array (with the module image)
// comes into being at the first call on a device, otherwise when the module
// loads: a caller whose pool reserves all free device memory makes that
// first call before reserving.  Host-side set-up uses small temporary heap
// buffers for the problem description; no device memory is allocated.
//
// The array is shared by all calls: each call clears the parts that must
// start at zero, and calls that overlap on the GPU (two streams, two host
// threads) race on it.  Its device address is looked up on every call with
// the caller's device current (cudaGetSymbolAddress), so a device reset or
// another current context never leaves a stale address behind; the first
// lookup on a device loads the module, so make the first call before any
// stream capture.
#include "../../include/vamp.h"
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using vamp::Params;
using vamp::Scalars;

namespace {

constexpr size_t VAMP_STATIC_SCRATCH_BYTES = size_t(8) << 20;  // 8 MiB

__device__ __align__(256) unsigned char g_scratch[VAMP_STATIC_SCRATCH_BYTES];

void put_msg(char* buf, int32_t len, const char* msg)
{
    if (buf && len > 0) {
        std::snprintf(buf, (size_t)len, "%s", msg);
    }
}

// Device address of the scratch array in the current context.  Looked up on
// every call (a table lookup once the module is loaded): an address cached
// per device ordinal would go stale after cudaDeviceReset or under another
// current context, where the module and its array are loaded anew.
cudaError_t scratch_ptr(unsigned char** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = (unsigned char*)p;
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
    Params pr{};
    vamp::Setup S;
    std::string why;
    if (cfg->stratified) {
        put_msg(err_msg, err_len, "the allocation-free pass samples by importance only (stratified = 0)");
        return VAMP_ERR_INVALID_ARG;
    }
    if (!vamp::build_setup(cfg, pr, S, why)) {
        put_msg(err_msg, err_len, ("invalid problem description: " + why).c_str());
        return VAMP_ERR_INVALID_ARG;
    }
    const int d = S.d, K = S.K, n = S.n;
    // bound n_calls before adding the per-channel minimum (no signed overflow)
    if (n_calls < 1 || iteration >= 0x80000000u || n_calls > int64_t(0xffffffff) ||
        n_calls > int64_t(0xffffffff) - (int64_t)K * cfg->n_min) {
        put_msg(err_msg, err_len, "n_calls must be >= 1, iteration < 2^31, total calls < 2^32");
        return VAMP_ERR_INVALID_ARG;
    }
    const int fp32 = S.fp32;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const vamp::Arena ar = vamp::plan_arena(pr);
    if (ar.bytes > VAMP_STATIC_SCRATCH_BYTES) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "problem needs %zu bytes of scratch; the static limit is %zu bytes", ar.bytes,
                      VAMP_STATIC_SCRATCH_BYTES);
        put_msg(err_msg, err_len, msg);
        return VAMP_ERR_INVALID_ARG;
    }
    int tile = 1;
    size_t smem = 0, smem_gen = 0;
    const std::vector<const vamp::PassVariant*> cand = vamp::pass_candidates(fp32, d, n);
    vamp::pass_smem_for(pr, fp32, cand.empty() ? 2 : cand[0]->minb, &tile, &smem, &smem_gen);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    unsigned char* base = nullptr;
    if (e == cudaSuccess) e = scratch_ptr(&base);
    int maxsm = 0, sms = 0, bps = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && ((int)smem > maxsm || cand.empty())) {
        put_msg(err_msg, err_len, "grid too large for shared memory");
        return VAMP_ERR_INVALID_ARG;
    }
    const vamp::PassVariant* var = e == cudaSuccess ? cand[0] : nullptr;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // raise (never lower) the kernel's dynamic shared-memory limit, which
    // contexts created with vamp_create may also rely on
    if (e == cudaSuccess) e = vamp::ensure_smem(var->fn[0], smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, var->fn[0], vamp::PASS_THREADS, smem);
    if (e != cudaSuccess) {
        put_msg(err_msg, err_len, cudaGetErrorString(e));
        return VAMP_ERR_CUDA;
    }
    vamp::bind_arena(pr, base, ar);
    pr.edges64 = const_cast<double*>(dev_edges);  // read only by the kernels launched here
    pr.alpha = const_cast<double*>(dev_alpha);    // read only by the kernels launched here
    const size_t rows = (size_t)K * d;
    // everything that must start from zero: accumulators and scalars
    e = cudaMemsetAsync(pr.D, 0, rows * n * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr.csum, 0, 2 * K * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr.sc, 0, sizeof(Scalars), stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pr.shift, dev_shift, K * 8, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = vamp::upload_setup(pr, S, stream);
    if (e == cudaSuccess) e = vamp::launch_derive(pr, stream);
    if (e == cudaSuccess) e = vamp::launch_begin_pass(pr, n_calls, stream);
    if (e == cudaSuccess) {
        vamp::PassArgs A{};
        A.field = iteration;
        A.tile = tile;
        A.ntiles = (K + tile - 1) / tile;
        e = var->launch(pr, 0, A, (bps > 0 ? bps : 1) * sms, smem, stream);
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

// vamp_peaks.cu -- vamp_measure_peaks: the per-pipe throughput of this GPU
// measured with small kernels, the denominators of the benchmark's
// per-pipe roofline (FP32 lanes, FP64 lanes, the MUFU special-function unit,
// shared-memory load wavefronts and L2 reads).
//
// Each kernel runs enough independent dependency chains per thread to keep
// its pipe busy, over a grid of every SM's resident CTAs, and is timed with
// CUDA events; the count of executed operations over the time is the peak.
#include "../../include/vamp.h"

#include <cuda_runtime.h>

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(float* out, float b, float c, int iters)
{
    float a[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int r = 0; r < iters; ++r)
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) a[i] = fmaf(a[i], b, c);
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(double* out, double b, double c, int iters)
{
    double a[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
    for (int r = 0; r < iters; ++r)
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) a[i] = fma(a[i], b, c);
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float v)
{
    float r;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// MUFU: x <- 2^x * c keeps x in (0, 1] for c = 0.5 (one FMUL per MUFU op,
// on the FMA pipe, which has eight times the MUFU rate)
__global__ void __launch_bounds__(PK_THREADS) k_peak_mufu(float* out, float c, int iters)
{
    float a[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) a[i] = (float)(threadIdx.x % 7 + i) * 0.1f;
    for (int r = 0; r < iters; ++r)
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) a[i] = ex2_approx(a[i]) * c;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

// Shared-memory loads: each warp reads 32 consecutive words (one wavefront
// per load instruction, no bank conflict)
constexpr int PK_SMEM_WORDS = 4096;
__global__ void __launch_bounds__(PK_THREADS) k_peak_lds(unsigned* out, int iters)
{
    __shared__ unsigned s[PK_SMEM_WORDS];
    for (int i = threadIdx.x; i < PK_SMEM_WORDS; i += PK_THREADS) s[i] = (unsigned)i * 2654435761u;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned acc[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) acc[i] = 0u;
    // chain i of step r reads row ((w + r) 8 + i) mod ROWS: rows come in
    // groups of eight, so one base register plus an immediate addresses
    // them (two instructions per load: the loads, not the issue rate, bind)
    constexpr int ROWS = PK_SMEM_WORDS / 32;
    for (int r = 0; r < iters; ++r) {
        const unsigned* rb = s + ((((w + r) * PK_CHAINS) & (ROWS - 1)) * 32 + lane);
#pragma unroll
        for (int i = 0; i < PK_CHAINS; ++i) acc[i] += rb[i * 32];
    }
    unsigned t = 0u;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) t ^= acc[i];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = t;
}

// L2 reads: coalesced 16-byte loads over a buffer that stays in L2 (the
// loads do not allocate in L1), PK_CHAINS independent loads per step
constexpr int PK_L2_LOG4 = 21;  // 2^21 float4 = 32 MiB
__device__ __forceinline__ float4 ld_l2(const float4* p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}
__global__ void __launch_bounds__(PK_THREADS) k_peak_l2(const float4* buf, float* out, int iters)
{
    const unsigned mask = (1u << PK_L2_LOG4) - 1u;
    const unsigned nt = gridDim.x * PK_THREADS;
    unsigned i = blockIdx.x * PK_THREADS + threadIdx.x;
    float s = 0.f;
    for (int r = 0; r < iters; ++r) {
        float4 v[PK_CHAINS];
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) v[c] = ld_l2(buf + ((i + c * nt) & mask));
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) s += (v[c].x + v[c].y) + (v[c].z + v[c].w);
        i += PK_CHAINS * nt;
    }
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

template <typename F>
cudaError_t time_kernel(F launch, float* ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    launch();  // warm-up
    e = cudaEventRecord(e0);
    if (e == cudaSuccess) launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

extern "C" vamp_status vamp_measure_peaks(vamp_pipe_peaks* out)
{
    if (!out) return VAMP_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return VAMP_ERR_CUDA;
    int bf = 0, bd = 0, bm = 0, bl = 0, b2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_peak_ffma, PK_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bd, k_peak_dfma, PK_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, k_peak_mufu, PK_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, k_peak_lds, PK_THREADS, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_peak_l2, PK_THREADS, 0) != cudaSuccess)
        return VAMP_ERR_CUDA;
    const int grid = sms * (bf > 0 ? bf : 1);
    const int gd = sms * (bd > 0 ? bd : 1), gm = sms * (bm > 0 ? bm : 1), gl = sms * (bl > 0 ? bl : 1);
    const int g2 = sms * (b2 > 0 ? b2 : 1);
    int maxg = grid;
    for (int g : {gd, gm, gl, g2}) maxg = g > maxg ? g : maxg;
    void* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)maxg * PK_THREADS * 8) != cudaSuccess) return VAMP_ERR_OOM;
    void* l2buf = nullptr;
    const size_t l2bytes = (size_t)16 << PK_L2_LOG4;
    if (cudaMalloc(&l2buf, l2bytes) != cudaSuccess) { cudaFree(buf); return VAMP_ERR_OOM; }
    vamp_status st = VAMP_OK;
    float ms = 0.f;
    const int it_f = 1 << 16, it_d = 1 << 12, it_m = 1 << 13, it_l = 1 << 14;
    cudaError_t e = time_kernel([&] { k_peak_ffma<<<grid, PK_THREADS>>>((float*)buf, 0.9999f, 1e-4f, it_f); }, &ms);
    if (e == cudaSuccess) out->fp32_lane_ops = (double)grid * PK_THREADS * PK_CHAINS * it_f / (ms * 1e-3);
    if (e == cudaSuccess)
        e = time_kernel([&] { k_peak_dfma<<<gd, PK_THREADS>>>((double*)buf, 0.9999, 1e-4, it_d); }, &ms);
    if (e == cudaSuccess) out->fp64_lane_ops = (double)gd * PK_THREADS * PK_CHAINS * it_d / (ms * 1e-3);
    if (e == cudaSuccess) e = time_kernel([&] { k_peak_mufu<<<gm, PK_THREADS>>>((float*)buf, 0.5f, it_m); }, &ms);
    if (e == cudaSuccess) out->xu_lane_ops = (double)gm * PK_THREADS * PK_CHAINS * it_m / (ms * 1e-3);
    if (e == cudaSuccess) e = time_kernel([&] { k_peak_lds<<<gl, PK_THREADS>>>((unsigned*)buf, it_l); }, &ms);
    if (e == cudaSuccess) out->lds_wavefronts = (double)gl * (PK_THREADS / 32) * PK_CHAINS * it_l / (ms * 1e-3);
    const int it_2 = 1 << 9;
    if (e == cudaSuccess) e = cudaMemset(l2buf, 0, l2bytes);
    if (e == cudaSuccess)
        e = time_kernel([&] { k_peak_l2<<<g2, PK_THREADS>>>((const float4*)l2buf, (float*)buf, it_2); }, &ms);
    if (e == cudaSuccess) out->l2_read_bytes = (double)g2 * PK_THREADS * PK_CHAINS * it_2 * 16.0 / (ms * 1e-3);
    if (e != cudaSuccess) st = VAMP_ERR_CUDA;
    cudaFree(buf);
    cudaFree(l2buf);
    return st;
}

// vamp_internal.h -- launch interface between the C ABI (vamp_api.cu) and
// the kernels (vamp_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vamp {

struct Params;

constexpr int PASS_THREADS = 256;  // threads per pass CTA
constexpr int CPT32 = 2;           // calls per thread, FP32-eval pass
constexpr int CPT64 = 1;           // calls per thread, FP64 pass
constexpr int SMEM_HEAD = 512;     // bytes of barriers and scratch before the tile buffers
constexpr int REFINE_WARPS = 4;    // grid rows per refine CTA

// Launch arguments of the pass kernel.  Integration: `field` = iteration.
// Generation: calls [0, batch) of stream `field`, in chunks of `chunk` =
// PASS_THREADS * CPT calls; accepted records of chunk b land in `staging`
// from slot b * chunk on, in call order.
struct PassArgs {
    uint32_t field;
    int tile;          // channels per staged tile
    int ntiles;        // ceil(K / tile)
    int rec_bytes;
    int64_t batch;
    int64_t chunk;
    int64_t nchunks;
    unsigned char* staging;   // [nchunks * chunk][rec_bytes]
    uint32_t* callidx;        // [nchunks * chunk]
    int* counts;              // [nchunks]
    long long* offsets;       // [nchunks]
};

struct EvalArgs {
    int mode;
    uint32_t field;
    uint32_t call0;
    int count;
    double* x;
    double* p;
    int* jf;
    int* bins;
    double* fgwc;
};

cudaError_t launch_begin_pass(const Params& P, int64_t N, cudaStream_t s);
const void* pass_kernel(int fp32, int mode);
cudaError_t launch_pass(const Params& P, int fp32, int mode, const PassArgs& A, int grid, size_t smem,
                        cudaStream_t s);
cudaError_t launch_finish_pass(const Params& P, int combine, cudaStream_t s);
cudaError_t launch_derive(const Params& P, cudaStream_t s);
cudaError_t launch_refine(const Params& P, cudaStream_t s);
cudaError_t launch_update_alpha(const Params& P, cudaStream_t s);
cudaError_t launch_gen_prepare(const Params& P, cudaStream_t s);
cudaError_t launch_gen_finish(const Params& P, const PassArgs& G, int64_t remaining, unsigned char* out,
                              cudaStream_t s);
cudaError_t launch_eval(const Params& P, int fp32, const EvalArgs& A, cudaStream_t s);

}  // namespace vamp

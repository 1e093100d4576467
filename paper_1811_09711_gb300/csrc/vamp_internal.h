// vamp_internal.h -- launch interface between the C ABI (vamp_api.cu) and
// the kernels (vamp_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vamp {

struct Params;

constexpr int SAMPLE_THREADS = 256;  // threads per sampling CTA
constexpr int REFINE_WARPS = 4;      // grid rows per refine CTA
constexpr int GEN_THREADS = 256;     // threads per generation CTA
constexpr int GEN_ROUNDS = 4;        // rounds of GEN_THREADS calls per generation CTA

// One generation batch: calls [0, batch) of stream `field`, processed in
// chunks of `chunk` calls per CTA; accepted records land in `staging` at
// the CTA's chunk offset, in call order.
struct GenArgs {
    uint32_t field;
    int64_t batch;
    int64_t chunk;
    int nblocks;
    int rec_bytes;
    unsigned char* staging;   // [batch][rec_bytes]
    uint32_t* callidx;        // [batch]
    int* counts;              // [nblocks]
    long long* offsets;       // [nblocks]
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
cudaError_t launch_sample(const Params& P, int fp32, uint32_t iteration, int grid, cudaStream_t s);
cudaError_t sample_occupancy(int fp32, int d, int n, int* blocks_per_sm);
cudaError_t launch_finish_pass(const Params& P, int combine, cudaStream_t s);
cudaError_t launch_derive(const Params& P, cudaStream_t s);
cudaError_t launch_refine(const Params& P, cudaStream_t s);
cudaError_t launch_update_alpha(const Params& P, cudaStream_t s);
cudaError_t launch_gen_prepare(const Params& P, cudaStream_t s);
cudaError_t launch_gen_batch(const Params& P, int fp32, const GenArgs& G, int64_t remaining,
                             unsigned char* out, cudaStream_t s);
cudaError_t launch_eval(const Params& P, int fp32, const EvalArgs& A, cudaStream_t s);

}  // namespace vamp

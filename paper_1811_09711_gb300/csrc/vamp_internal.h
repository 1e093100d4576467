// vamp_internal.h -- interface between the C ABI (vamp_api.cu,
// vamp_noalloc.cu), the host-side setup (vamp_setup.cu) and the kernels.
// Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/vamp.h"

namespace vamp {

struct Params;
template <typename T> struct MapRec;

constexpr int PASS_THREADS = 256;  // threads per pass CTA (PASS_THREADS_DEV in the device code)
constexpr int SMEM_HEAD = 512;     // bytes of barriers and scratch before the tile buffers
constexpr int REFINE_WARPS = 4;    // grid rows per refine CTA
constexpr size_t TILE_BUDGET = 112 * 1024;  // pass-kernel shared memory per CTA (two CTAs per SM)

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

// One compiled pass kernel pair (integration, generation): precision, calls
// per thread, and the shape it is specialised for (D = NB = 0: any shape).
struct PassVariant {
    int fp32, cpt, D, NB;
    int minb;  // CTAs per SM the kernel is compiled for (register cap), sizes its tile budget
    const char* family;  // kernel template name ("k_pass" or "k_union")
    int uni = 0;         // runs on the union interval tables (vamp_union.cu), not on staged tiles
    const void* fn[2];
    cudaError_t (*launch)(const Params& P, int mode, const PassArgs& A, int grid, size_t smem, cudaStream_t s);
};

void add_pass_variants_f32_generic(std::vector<PassVariant>& v);
void add_pass_variants_f32_shapes(std::vector<PassVariant>& v);
void add_pass_variants_f64(std::vector<PassVariant>& v);
void add_pass_variants_union(std::vector<PassVariant>& v);

// ---- interval tables of the union pass (vamp_union.cu) -----------------------
// Whether the union kernels take a problem of this kind: FP32-eval,
// importance sampling, K <= UNION_SLOTS and K (n+1) <= UNION_MAXV.
bool union_fits(int fp32, int d, int K, int n, int stratified);
size_t union_bytes(int d, int K, int n);           // device bytes of the tables
void bind_union(Params& P, unsigned char* base);   // sets P.u* (null: no tables)
// Rebuilds the tables from P's master grids and lookup blocks (enqueued on s).
cudaError_t launch_union_build(const Params& P, cudaStream_t s);
size_t union_pass_smem(const Params& P, const PassVariant& v, int mode);

// Host-side data derived from a vamp_config (vamp_setup.cu).
struct Setup {
    int d = 0, K = 0, n = 0, P = 0, fp32 = 0;
    double zinv = 1.0;
    std::vector<unsigned char> hdr64, hdr32;  // K lookup-block headers each
    std::vector<unsigned char> pk64, pk32;    // P MapRec records each (non-matching integrand)
    std::vector<int32_t> eq_off, eq_ent;      // channel equivalences by grid row (Params::eq_off)
};

// Validates cfg, fills the scalar fields of P (keys, layouts, Gaussian,
// matching flag) and the host images in S.  Returns false with a reason.
bool build_setup(const vamp_config* cfg, Params& P, Setup& S, std::string& why);

// Device-side placement of the per-problem arrays inside one buffer.
struct Arena {
    size_t edges64, lk64, lk32, alpha, alpha32, shift, acum, nc, pc, D, csum, ic, vc, wc, pk64, pk32, sc;
    size_t nr, spc, coff, qc;
    size_t eqoff, eqent;   // 0 bytes without equivalences
    size_t bytes;
};
Arena plan_arena(const Params& P);
void bind_arena(Params& P, unsigned char* base, const Arena& A);  // sets every array pointer
// Copies headers and peak records into the arena (async on s).
cudaError_t upload_setup(const Params& P, const Setup& S, cudaStream_t s);

// Tile and shared-memory size of the pass kernel: two CTAs per SM
// (TILE_BUDGET), or `minb` CTAs per SM of the current device.
void pass_smem(const Params& P, int fp32, int* tile, size_t* smem_int, size_t* smem_gen);
void pass_smem_for(const Params& P, int fp32, int minb, int* tile, size_t* smem_int, size_t* smem_gen);
// Candidate kernels for a shape: exact (D, NB) matches first, then generic;
// with the channel count K given (K > 0) and union_fits, the union kernels
// after them (exact shape first).
std::vector<const PassVariant*> pass_candidates(int fp32, int d, int n, int stratified = 0, int K = 0);
// Raises (never lowers) the dynamic shared-memory limit of a kernel.
cudaError_t ensure_smem(const void* fn, size_t bytes);

// ---- many instances in one launch -------------------------------------------
// Per-iteration arguments read by the batch kernels (copied from pinned host
// memory by the first node of the iteration graph).
struct BatchIter {
    uint32_t iteration;
    int32_t adapt;         // bit 0: refine grids, bit 1: update α
};
// Work-item bookkeeping of the multi-instance pass kernel.
struct BatchCtl {
    long long total;       // work items of this iteration
    long long next;        // next item to hand out (atomic)
};
struct MultiArgs {
    const Params* inst;          // [n] instance parameters
    const int* tiles;            // [n] channels per staged tile
    const int* combine_from;     // [n]
    const int64_t* ncalls;       // [n] calls requested this iteration
    const uint32_t* iter;        // [n] iteration index (random stream) of each instance
    const int* pair_off;         // [n+1] first (instance, channel) pair of instance i
    long long* pair_prefix;      // [npairs+1] items before each pair
    const int* row_off;          // [n+1] first grid row of instance i (rows = K*d)
    BatchCtl* ctl;
    const BatchIter* it;
    double* results;             // [n][9]: pass result (8) and calls
    int n_inst;
    int npairs;
    int nrows;
    int max_n;                   // largest bins per axis
    int64_t item_calls;          // calls per work item (multiple of PASS_THREADS*CPT)
    int any_strat;               // some instance samples pseudo-stratified (its own kernel form)
};
constexpr int PARAMS_SLOT = 512;  // bytes reserved for an instance's Params in shared memory

cudaError_t launch_batch_begin(const MultiArgs& M, cudaStream_t s);
cudaError_t launch_batch_after(const MultiArgs& M, cudaStream_t s);  // finish, refine, α, gather
// minb: CTAs per SM the kernel is compiled for (2, or 3 in the FP32-eval form)
cudaError_t launch_pass_multi(int fp32, int minb, const MultiArgs& M, int grid, size_t smem, cudaStream_t s);
// strat: the form that also runs pseudo-stratified instances
const void* pass_multi_kernel(int fp32, int minb, int strat = 0);

cudaError_t launch_begin_pass(const Params& P, int64_t N, cudaStream_t s);
cudaError_t launch_finish_pass(const Params& P, int combine, cudaStream_t s);
cudaError_t launch_strat_q(const Params& P, cudaStream_t s);  // stratified passes, before finish
cudaError_t launch_derive(const Params& P, cudaStream_t s);
cudaError_t launch_refine(const Params& P, cudaStream_t s);
cudaError_t launch_update_alpha(const Params& P, cudaStream_t s);
cudaError_t launch_pass_result(const Params& P, double* out, cudaStream_t s);  // 9 doubles
cudaError_t launch_gen_prepare(const Params& P, cudaStream_t s);
cudaError_t launch_gen_finish(const Params& P, const PassArgs& G, int64_t remaining, unsigned char* out,
                              cudaStream_t s);
cudaError_t launch_eval(const Params& P, int fp32, const EvalArgs& A, cudaStream_t s);
cudaError_t launch_wait_selftest(long long limit, unsigned int* flag, long long* cycles, cudaStream_t s);

}  // namespace vamp

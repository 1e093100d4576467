// vamp_batch_pass.cu -- one persistent pass kernel for many independent
// integrations of uneven dimension, channel count, bins and call count.
//
// The iteration's work is cut into items: item = up to `item_calls`
// consecutive calls of one channel of one instance (so that the item's
// d-value accumulators in shared memory belong to one (instance, channel)).
// Persistent CTAs take items from an atomic counter until none are left; for
// each item a CTA copies the instance's parameters into shared memory,
// streams that instance's channel tiles through the two bulk-copy buffers
// and runs the same three phases as the single-instance pass kernel.  No CTA
// waits on another CTA: the counter is the only shared state.
//
// The item code is compiled for four dimension classes (d in 1..4, 5..8,
// 9..12, 13..16): each unrolls its row loops to the class's largest d with
// no test on the rows every member has, and the classes of small d process
// two calls per thread.
#include "vamp_pass.cuh"

namespace vamp {

// Barrier bookkeeping of a CTA across items: use v of an item lives in
// buffer v%2 (streaming) or v, at phase done_b + v/2 (or 0).
struct ItemPipe {
    uint32_t done0 = 0u, done1 = 0u;
};

// One work item: calls [a, b) of channel c of the instance in Ps.  Returns
// false if a bounded wait gave up (the CTA then drains and exits).
template <typename T, int CPT, class SH>
__device__ __forceinline__ bool run_item(const MultiArgs& M, const Params& P, SmemHead& H, unsigned char* buf0,
                                         int inst, int c, long long kth, ItemPipe& pp, bool& bad)
{
    constexpr int B = PASS_THREADS * CPT;
    const int tid = threadIdx.x;
    const SH sh(Prec<T>::lay(P), P.d, P.n);
    const int tile = M.tiles[inst];
    const int ntiles = (P.K + tile - 1) / tile;
    const int S = sh.bytes();
    const size_t tile_bytes = (size_t)tile * S;
    double* Ds = reinterpret_cast<double*>(buf0 + 2 * tile_bytes);
    const int dn = P.d * P.n;
    const int64_t a = P.Pc[c] + kth * M.item_calls;
    const int64_t b = min(a + M.item_calls, (int64_t)P.Pc[c + 1]);
    const int64_t nb = (b - a + B - 1) / B;
    const bool streaming = ntiles > 2;
    const int64_t total_uses = streaming ? nb * ntiles : ntiles;
    const unsigned char* lk = Prec<T>::lk(P);
    auto issue = [&](int64_t u) {
        const int t = (int)(u % ntiles);
        const int cnt = min(tile, P.K - t * tile);
        fence_proxy_async_smem();
        bulk_load(buf0 + (u & 1) * tile_bytes, lk + (size_t)t * tile_bytes, (uint32_t)(cnt * S), &H.bar[u & 1]);
    };
    for (int q = tid; q < dn; q += PASS_THREADS) Ds[q] = 0.0;
    __syncthreads();
    if (tid == 0) {
        issue(0);
        if (total_uses > 1) issue(1);
    }
    int64_t u = 0, issued = total_uses > 1 ? 2 : 1;
    double s1 = 0.0, s2 = 0.0, wm = 0.0;
    const double sft = P.shift[c];
    for (int64_t bt = 0; bt < nb; ++bt) {
        const int64_t base = a + bt * B, end = min(b, base + B);
        Calls<T, CPT, SH::DM> C;
        phase_a<T, 0, CPT>(P, sh, M.iter[inst], base, end, c, C);
        for (int t = 0; t < ntiles; ++t) {
            const int bb = streaming ? (int)(u & 1) : t;
            if (streaming || bt == 0) {
                const uint32_t ph = (bb ? pp.done1 : pp.done0) + (streaming ? (uint32_t)(u >> 1) : 0u);
                if (!mbar_wait_bounded(&H.bar[bb], ph & 1u)) {
                    atomicOr(&P.sc->err, ERR_TIMEOUT);
                    H.abort = 1;
                }
            }
            if (!H.abort) tile_compute<T, 0, CPT>(P, sh, buf0 + bb * tile_bytes, t, tile, c, C);
            __syncthreads();
            if (H.abort) {
                // let this CTA's copies in flight land (bounded), then give up
                if (tid == 0) {
                    for (int64_t v = u; v < issued; ++v) {
                        const int vb = streaming ? (int)(v & 1) : (int)v;
                        const uint32_t ph = (vb ? pp.done1 : pp.done0) + (streaming ? (uint32_t)(v >> 1) : 0u);
                        mbar_wait_bounded(&H.bar[vb], ph & 1u);
                    }
                }
                __syncthreads();
                return false;
            }
            if (streaming && tid == 0 && issued < total_uses) {
                issue(issued);
                ++issued;
            }
            ++u;
        }
        phase_c_int<T, CPT>(sh, C, sft, Ds, s1, s2, wm, bad,
                            (SH::kStrat && P.stratified) ? CellSums{P.cellsum, base - P.Pc[c], P.spc[c], P.coff[c]}
                                                         : CellSums{nullptr, 0, 1, 0});
    }
    // uses of each buffer in this item
    if (streaming) {
        pp.done0 += (uint32_t)((total_uses + 1) / 2);
        pp.done1 += (uint32_t)(total_uses / 2);
    } else {
        pp.done0 += 1u;
        pp.done1 += ntiles > 1 ? 1u : 0u;
    }
    flush_segment(P, H, c, dn, Ds, s1, s2);
    block_max_to(H, wm, &P.sc->wmax_bits);
    return true;
}

template <typename T, int MINB, bool STRAT>
__global__ void __launch_bounds__(PASS_THREADS, MINB) k_pass_multi(MultiArgs M)
{
    static_assert(sizeof(Params) <= PARAMS_SLOT, "Params does not fit its shared-memory slot");
    extern __shared__ __align__(128) unsigned char smem[];
    SmemHead& H = *reinterpret_cast<SmemHead*>(smem);
    Params& Ps = *reinterpret_cast<Params*>(smem + SMEM_HEAD);
    unsigned char* buf0 = smem + SMEM_HEAD + PARAMS_SLOT;
    __shared__ long long s_item;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&H.bar[0], 1);
        mbar_init(&H.bar[1], 1);
        H.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    ItemPipe pp;
    int cur = -1;
    bool bad = false;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&M.ctl->next), 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= M.ctl->total) break;
        // (instance, channel, k-th item of the pair)
        int lo = 0, hi = M.npairs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (M.pair_prefix[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int pair = lo;
        lo = 0;
        hi = M.n_inst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (M.pair_off[mid] <= pair) lo = mid; else hi = mid - 1;
        }
        const int inst = lo;
        const int c = pair - M.pair_off[inst];
        const long long kth = item - M.pair_prefix[pair];
        if (inst != cur) {
            const int* src = reinterpret_cast<const int*>(&M.inst[inst]);
            int* dst = reinterpret_cast<int*>(&Ps);
            for (int q = tid; q < (int)(sizeof(Params) / sizeof(int)); q += PASS_THREADS) dst[q] = src[q];
            cur = inst;
        }
        __syncthreads();
        const int d = Ps.d;
        bool ok;
        // pseudo-stratified instances: the generic shape, which carries the
        // cell digits and cell sums (compiled only into the STRAT form)
        if (STRAT && Ps.stratified) ok = run_item<T, 1, Shape<T, 0, 0>>(M, Ps, H, buf0, inst, c, kth, pp, bad);
        else if (d <= 4) ok = run_item<T, 2, Shape<T, 0, 0, 4, 1>>(M, Ps, H, buf0, inst, c, kth, pp, bad);
        else if (d <= 8) ok = run_item<T, 2, Shape<T, 0, 0, 8, 5>>(M, Ps, H, buf0, inst, c, kth, pp, bad);
        else if (d <= 12) ok = run_item<T, 1, Shape<T, 0, 0, 12, 9>>(M, Ps, H, buf0, inst, c, kth, pp, bad);
        else ok = run_item<T, 1, Shape<T, 0, 0, 16, 13>>(M, Ps, H, buf0, inst, c, kth, pp, bad);
        if (!ok) return;
        if (bad) {
            atomicOr(&Ps.sc->err, ERR_NONFINITE);
            bad = false;
        }
        __syncthreads();
    }
}

// Compiled for two or (FP32-eval) three CTAs per SM.
const void* pass_multi_kernel(int fp32, int minb, int strat)
{
    if (strat) {
        if (!fp32) return (const void*)k_pass_multi<double, 2, true>;
        return minb >= 3 ? (const void*)k_pass_multi<float, 3, true> : (const void*)k_pass_multi<float, 2, true>;
    }
    if (!fp32) return (const void*)k_pass_multi<double, 2, false>;
    return minb >= 3 ? (const void*)k_pass_multi<float, 3, false> : (const void*)k_pass_multi<float, 2, false>;
}

cudaError_t launch_pass_multi(int fp32, int minb, const MultiArgs& M, int grid, size_t smem, cudaStream_t s)
{
    if (M.any_strat) {
        if (!fp32) k_pass_multi<double, 2, true><<<grid, PASS_THREADS, smem, s>>>(M);
        else if (minb >= 3) k_pass_multi<float, 3, true><<<grid, PASS_THREADS, smem, s>>>(M);
        else k_pass_multi<float, 2, true><<<grid, PASS_THREADS, smem, s>>>(M);
    } else {
        if (!fp32) k_pass_multi<double, 2, false><<<grid, PASS_THREADS, smem, s>>>(M);
        else if (minb >= 3) k_pass_multi<float, 3, false><<<grid, PASS_THREADS, smem, s>>>(M);
        else k_pass_multi<float, 2, false><<<grid, PASS_THREADS, smem, s>>>(M);
    }
    return cudaGetLastError();
}

}  // namespace vamp

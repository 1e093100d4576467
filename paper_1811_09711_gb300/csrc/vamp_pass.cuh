// vamp_pass.cuh -- the persistent pass kernel, templated on precision, mode
// (0 integration, 1 generation), calls per thread and problem shape.
//
// Each CTA owns a contiguous range of calls (integration: split further at
// channel boundaries so that its d-value accumulators in shared memory
// belong to one channel) or a strided set of call chunks (generation), and
// processes them in batches of PASS_THREADS*CPT calls:
//   A  per call: Philox words, channel (integration: the segment's; generation:
//      drawn from α), forward map x_c -> p on the channel's grid, its own term
//      α_c g_c/φ'_c of g(p), Gaussian exponent sum (and the integrand when the
//      peaks are not the channels' maps);
//   B  every channel's term of g(p) (Eq. 30) and the matching integrand peak,
//      with the channels' lookup blocks streamed through shared memory in
//      tiles (cp.async.bulk, two buffers, bounded mbarrier waits);
//   C  w = f/g: per-channel shifted sums, d-values D_{c,k,j} += w² (Eq. 15),
//      max |weight| (integration); accept u w_max < |w| and ordered compaction
//      of the event records (generation).
#pragma once

#include "vamp_device.cuh"
#include "vamp_internal.h"

namespace vamp {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

static_assert(PASS_THREADS == PASS_THREADS_DEV, "device copy of the CTA size");

struct SmemHead {
    uint64_t bar[2];
    int abort;
    int pad;
    double red[3][PASS_THREADS / 32];
    int wcnt[PASS_THREADS / 32];
    int woff[PASS_THREADS / 32];
    int round_total;
};
static_assert(sizeof(SmemHead) <= SMEM_HEAD, "shared-memory head too large");

// Per-thread state of the CPT calls of one batch.
template <typename T, int CPT, int DM>
struct Calls {
    T p[CPT][DM], g[CPT], f[CPT], Aexp[CPT];
    bool valid[CPT];
    int cq[CPT];
    uint32_t jp[CPT][(DM + 3) / 4];
    uint32_t xacc[CPT];
};

// Cell sums of a stratified batch: the call at local index l (from the
// channel's first call) belongs to cell coff + l / spc.
struct CellSums {
    double* sum;     // nullptr: importance sampling
    int64_t l0;      // local index of the batch's first call
    int64_t spc;     // calls per cell
    int64_t coff;    // first cell of the channel
};

// Phase A: Philox words, channel, forward map on the channel's grid, own
// term of g(p), Gaussian exponent sum; the integrand when peaks are not the
// channels' maps.  Call q of this thread is base + q*PASS_THREADS + tid.
template <typename T, int MODE, int CPT, class SH>
__device__ __forceinline__ void phase_a(const Params& P, const SH& sh, uint32_t field, int64_t base, int64_t end,
                                        int cseg, Calls<T, CPT, SH::DM>& C)
{
    constexpr int DM = SH::DM;
    const int d = sh.d();
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int64_t i = base + (int64_t)q * PASS_THREADS + tid;
        C.valid[q] = i < end;
        uint32_t X[DM + 4];
        call_words<DM + 4>(P, (uint32_t)(C.valid[q] ? i : base), field, MODE == 0 ? d : d + 2, X);
        int c;
        if (MODE == 0) {
            c = cseg;
            C.xacc[q] = 0u;
        } else {
            uint32_t xc = 0u, xa = 0u;
#pragma unroll
            for (int k = 0; k < DM + 4; ++k) {
                if (k == d) xc = X[k];
                if (k == d + 1) xa = X[k];
            }
            c = choose_channel(P, unif64(xc));
            C.xacc[q] = xa;
        }
        C.cq[q] = c;
        T x[DM];
        int jf[DM];
        T owngJ, Aq;
        if (MODE == 0 && SH::kStrat && P.stratified) {
            // cell of the call and its base-n_r digits (§3.3)
            const uint32_t nr = (uint32_t)P.nr[c];
            uint32_t cell = (uint32_t)(((C.valid[q] ? i : base) - P.Pc[c]) / P.spc[c]);
            uint32_t dig[DM];
#pragma unroll
            for (int k = 0; k < DM; ++k) {
                dig[k] = cell % nr;
                cell /= nr;
            }
            forward_call<T>(P, sh, c, X, x, C.p[q], jf, owngJ, Aq, dig, nr);
        } else {
            forward_call<T>(P, sh, c, X, x, C.p[q], jf, owngJ, Aq);
        }
        C.Aexp[q] = Aq;
#pragma unroll
        for (int w = 0; w < (DM + 3) / 4; ++w) {
            uint32_t v = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (4 * w + b < DM) v |= (uint32_t)(jf[4 * w + b] & 0xff) << (8 * b);
            C.jp[q][w] = v;
        }
        C.g[q] = Prec<T>::alpha(P, c) * owngJ;
        C.f[q] = P.matching ? T(0) : integrand_peaks<T, DM>(P, d, C.p[q], Aq);
    }
}

// Phase B for one staged tile: channels t*tile .. of the tile buffer tb.
template <typename T, int MODE, int CPT, class SH>
__device__ __forceinline__ void tile_compute(const Params& P, const SH& sh, const unsigned char* tb, int t, int tile,
                                             int cseg, Calls<T, CPT, SH::DM>& C, const T* pw = nullptr)
{
    const int S = sh.bytes();
    const int cnt = min(tile, P.K - t * tile);
    bool skip[CPT];
    for (int cl = 0; cl < cnt; ++cl) {
        const int c2 = t * tile + cl;
        const T a = Prec<T>::alpha(P, c2);
        const bool lookups = (a != T(0)) && !(MODE == 0 && c2 == cseg);
#pragma unroll
        for (int q = 0; q < CPT; ++q) skip[q] = (MODE == 1) && (C.cq[q] == c2);
        channel_body<T, CPT, false>(P, sh, tb + (size_t)cl * S, a, lookups, P.matching != 0, C.p, C.Aexp, skip,
                                    C.g, C.f, nullptr, pw);
    }
}

// Word i of a small register array, by a chain of selects (no local memory).
template <int W>
__device__ __forceinline__ uint32_t pick(const uint32_t (&a)[W], int i)
{
    uint32_t v = a[0];
#pragma unroll
    for (int t = 1; t < W; ++t) v = i == t ? a[t] : v;
    return v;
}

// Phase C of an integration batch: shifted sums, max weight and the d-values
// (Eq. 15) of the segment's channel in shared memory (FP64 atomics, which
// retry on collisions).  Unless the shape has many bins per axis (a lane's
// bins then rarely collide), lane l adds its d terms in the rotated axis
// order l, l+1, ... (mod d), so that at any step the lanes of a warp hit
// different rows.
template <typename T, int CPT, class SH>
__device__ __forceinline__ void phase_c_int(const SH& sh, const Calls<T, CPT, SH::DM>& C, double sft, double* Ds,
                                            double& s1, double& s2, double& wm, bool& bad,
                                            const CellSums cs = CellSums{nullptr, 0, 1, 0})
{
    constexpr int DM = SH::DM;
    const int d = sh.d(), n = sh.n();
    constexpr bool kRotate = !(SH::kN && SH::NBC >= 64);
    const int rot = kRotate ? (threadIdx.x & 31) % d : 0;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        if (!C.valid[q]) continue;
        double w = C.g[q] > T(0) ? (double)(C.f[q] / C.g[q]) : 0.0;
        if (!isfinite(w)) { bad = true; w = 0.0; }
        const double dv = w - sft;
        s1 += dv;
        s2 += dv * dv;
        if (cs.sum)  // stratified: the sum of the call's cell
            atomicAdd(&cs.sum[cs.coff + (cs.l0 + q * PASS_THREADS + (int)threadIdx.x) / cs.spc], dv);
        wm = fmax(wm, fabs(w));  // signed integrands: w_max bounds |w|
        const double w2 = w * w;
#pragma unroll
        for (int s = 0; s < DM; ++s) {
            if (sh.has(s)) {
                if (kRotate) {
                    int k = s + rot;
                    if (k >= d) k -= d;
                    const int j = (pick(C.jp[q], k >> 2) >> (8 * (k & 3))) & 0xff;
                    atomicAdd(&Ds[k * n + j], w2);
                } else {
                    atomicAdd(&Ds[s * n + ((C.jp[q][s >> 2] >> (8 * (s & 3))) & 0xff)], w2);
                }
            }
        }
    }
}

// Phase C of a generation batch (chunk `chunk`, calls from `base`): accept iff
// u w_max < |w| and write the accepted records of the chunk in call order
// (ballot within a warp, warp offsets through shared memory), then the
// chunk's count.  Every thread of the CTA takes part.
template <typename T, int CPT, class SH>
__device__ __forceinline__ void phase_c_gen(const Params& P, const PassArgs& A, const SH& sh,
                                            const Calls<T, CPT, SH::DM>& C, int64_t chunk, int64_t base,
                                            int* wcnt, int* woff, int* round_total, double& wm, bool& bad)
{
    constexpr int DM = SH::DM;
    constexpr int B = PASS_THREADS * CPT;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double wmax = P.sc->wmax_gen;
    int running = 0;
    const int64_t cbase = chunk * B;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        double w = 0.0;
        bool acc = false;
        if (C.valid[q]) {
            w = C.g[q] > T(0) ? (double)(C.f[q] / C.g[q]) : 0.0;
            if (!isfinite(w)) { bad = true; w = 0.0; }
            wm = fmax(wm, fabs(w));
            acc = unif64(C.xacc[q]) * wmax < fabs(w);  // the event keeps the sign of w
        }
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        if (lane == 0) wcnt[wid] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
            int s = 0;
            for (int w2 = 0; w2 < PASS_THREADS / 32; ++w2) { woff[w2] = s; s += wcnt[w2]; }
            *round_total = s;
        }
        __syncthreads();
        if (acc) {
            const int pos = running + woff[wid] + __popc(bal & ((1u << lane) - 1u));
            const int64_t slot = cbase + pos;
            // record {float p[d]; zero pad to 8 bytes; double w}: 8-byte
            // stores (records are 8-byte multiples at 8-byte offsets)
            unsigned char* rec = A.staging + slot * A.rec_bytes;
            float2* pf2 = reinterpret_cast<float2*>(rec);
#pragma unroll
            for (int k = 0; k < DM; k += 2)
                if (sh.has(k))
                    pf2[k >> 1] = make_float2((float)C.p[q][k],
                                              (k + 1 < DM && sh.has(k + 1)) ? (float)C.p[q][k + 1] : 0.0f);
            *reinterpret_cast<double*>(rec + A.rec_bytes - 8) = w;
            A.callidx[slot] = (uint32_t)(base + (int64_t)q * PASS_THREADS + tid);
        }
        running += *round_total;
        __syncthreads();
    }
    if (tid == 0) A.counts[chunk] = running;
}

// Flush of a segment: block sums of (s1, s2) and the d-values to global.
__device__ __forceinline__ void flush_segment(const Params& P, SmemHead& H, int cseg, int dn, double* Ds, double s1,
                                              double s2)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) { H.red[0][wid] = s1; H.red[1][wid] = s2; }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, bb = 0.0;
        for (int q = 0; q < PASS_THREADS / 32; ++q) { a += H.red[0][q]; bb += H.red[1][q]; }
        atomicAdd(&P.csum[2 * cseg], a);
        atomicAdd(&P.csum[2 * cseg + 1], bb);
    }
    double* Dg = P.D + (size_t)cseg * dn;
    for (int q = tid; q < dn; q += PASS_THREADS) {
        const double v = Ds[q];
        if (v != 0.0) atomicAdd(&Dg[q], v);
    }
    __syncthreads();
}

// Block maximum of wm into *dst (non-negative doubles compare as bits).
__device__ __forceinline__ void block_max_to(SmemHead& H, double wm, unsigned long long* dst)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    wm = warp_max(wm);
    if (lane == 0) H.red[2][wid] = wm;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int q = 0; q < PASS_THREADS / 32; ++q) m = fmax(m, H.red[2][q]);
        atomicMax(dst, (unsigned long long)__double_as_longlong(m));
    }
}

template <typename T, int MODE, int CPT, int D_, int NB_, int MINB>
__global__ void __launch_bounds__(PASS_THREADS, MINB) k_pass(Params P, PassArgs A)
{
    using SH = Shape<T, D_, NB_>;
    constexpr int DM = SH::DM;
    extern __shared__ __align__(128) unsigned char smem[];
    SmemHead& H = *reinterpret_cast<SmemHead*>(smem);
    unsigned char* buf0 = smem + SMEM_HEAD;
    const SH sh(Prec<T>::lay(P), P.d, P.n);
    const int S = sh.bytes();
    const size_t tile_bytes = (size_t)A.tile * S;
    double* Ds = reinterpret_cast<double*>(buf0 + 2 * tile_bytes);
    const int d = sh.d(), n = sh.n(), dn = d * n, K = P.K;
    const int tid = threadIdx.x;
    constexpr int B = PASS_THREADS * CPT;
    const unsigned char* lk = Prec<T>::lk(P);
    // FP64: the power-law Jacobian 0.2 p_k^(-4/5) of each coordinate of this
    // thread's call, computed once per call instead of once per channel that
    // maps k (after the tiles and the d-values; DMAX x PASS_THREADS doubles
    // are reserved by smem_for_budget)
    constexpr bool kPW = sizeof(T) == 8 && CPT == 1;
    T* pwS = nullptr;
    if constexpr (kPW) {
        // used only where the launch reserved the space (see smem_for_budget)
        unsigned dsm = 0;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
        const size_t off = SMEM_HEAD + 2 * tile_bytes + (MODE == 0 ? (size_t)dn * 8 : 0);
        if ((size_t)dsm >= off + (size_t)DM * PASS_THREADS * sizeof(T))
            pwS = reinterpret_cast<T*>(smem + off);
    }

    // ---- work of this CTA ---------------------------------------------------
    int64_t r0 = 0, r1 = 0;
    int64_t nbatch = 0;
    if (MODE == 0) {
        const int64_t N = P.sc->n_total;
        r0 = N * blockIdx.x / gridDim.x;
        r1 = N * (blockIdx.x + 1) / gridDim.x;
        int64_t i = r0;
        while (i < r1) {
            const int c = find_channel(P.Pc, K, i);
            const int64_t e = min(r1, P.Pc[c + 1]);
            nbatch += (e - i + B - 1) / B;
            i = e;
        }
    } else {
        const int64_t nch = A.nchunks;
        nbatch = blockIdx.x < nch ? (nch - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    }
    if (nbatch == 0) return;
    const int ntiles = A.ntiles;
    const bool streaming = ntiles > 2;
    const int64_t total_uses = streaming ? nbatch * ntiles : ntiles;

    auto issue = [&](int64_t u) {
        const int t = (int)(u % ntiles);
        const int cnt = min(A.tile, K - t * A.tile);
        fence_proxy_async_smem();
        bulk_load(buf0 + (u & 1) * tile_bytes, lk + (size_t)t * tile_bytes, (uint32_t)(cnt * S), &H.bar[u & 1]);
    };
    if (tid == 0) {
        mbar_init(&H.bar[0], 1);
        mbar_init(&H.bar[1], 1);
        H.abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        issue(0);
        if (total_uses > 1) issue(1);
    }
    int64_t u = 0;              // next tile use to consume
    int64_t issued = total_uses > 1 ? 2 : 1;
    double wm = 0.0, s1 = 0.0, s2 = 0.0;
    bool bad = false;

    // integration segment state
    int64_t i0 = r0;
    int cseg = -1;
    int64_t seg_end = 0;
    double sft = 0.0;
    // generation chunk state
    int64_t chunk = blockIdx.x;

    for (int64_t bt = 0; bt < nbatch; ++bt) {
        int64_t base, end;
        if (MODE == 0) {
            if (i0 >= seg_end || cseg < 0) {
                // new segment of one channel: reset the shared d-values
                cseg = find_channel(P.Pc, K, i0);
                seg_end = min(r1, P.Pc[cseg + 1]);
                sft = P.shift[cseg];
                for (int q = tid; q < dn; q += PASS_THREADS) Ds[q] = 0.0;
                s1 = s2 = 0.0;
                __syncthreads();
            }
            base = i0;
            end = min(seg_end, i0 + B);
        } else {
            base = chunk * B;
            end = min(A.batch, base + B);
        }

        // ---- phase A: own channel forward map, integrand --------------------
        Calls<T, CPT, DM> C;
        phase_a<T, MODE, CPT>(P, sh, A.field, base, end, cseg, C);
        if constexpr (kPW) {
            if (pwS) {
#pragma unroll
                for (int k = 0; k < DM; ++k) {
                    if (sh.has(k)) {
                        const T y = Prec<T>::rinv5(C.p[0][k]), y2 = y * y;
                        pwS[k * PASS_THREADS + tid] = T(0.2) * (y2 * y2);
                    }
                }
            }
        }

        // ---- phase B: every channel's term of g(p) (and the matching peaks) --
        for (int t = 0; t < ntiles; ++t) {
            // streaming: use u lives in buffer u%2 (phase u/2); otherwise tile t
            // stays in buffer t after the first batch
            const int b = streaming ? (int)(u & 1) : t;
            if (streaming || bt == 0) {
                if (!mbar_wait_bounded(&H.bar[b], streaming ? (uint32_t)((u >> 1) & 1) : 0u)) {
                    atomicOr(&P.sc->err, ERR_TIMEOUT);
                    H.abort = 1;
                }
            }
            if (!H.abort)
                tile_compute<T, MODE, CPT>(P, sh, buf0 + b * tile_bytes, t, A.tile, cseg, C, pwS ? pwS + tid : nullptr);
            __syncthreads();
            if (H.abort) goto drain;
            if (streaming && tid == 0 && issued < total_uses) {
                issue(issued);
                ++issued;
            }
            ++u;
        }

        // ---- phase C: weights and accumulation ------------------------------
        if (MODE == 0) {
            phase_c_int<T, CPT>(sh, C, sft, Ds, s1, s2, wm, bad,
                                (SH::kStrat && P.stratified)
                                    ? CellSums{P.cellsum, base - P.Pc[cseg], P.spc[cseg], P.coff[cseg]}
                                    : CellSums{nullptr, 0, 1, 0});
            i0 = end;
            if (i0 >= seg_end) {
                // end of the segment: flush its sums and d-values
                flush_segment(P, H, cseg, dn, Ds, s1, s2);
                s1 = s2 = 0.0;
            }
        } else {
            phase_c_gen<T, CPT>(P, A, sh, C, chunk, base, H.wcnt, H.woff, &H.round_total, wm, bad);
            chunk += gridDim.x;
        }
    }

    // ---- CTA totals --------------------------------------------------------
    if (bad) atomicOr(&P.sc->err, ERR_NONFINITE);
    block_max_to(H, wm, MODE == 0 ? &P.sc->wmax_bits : &P.sc->gen_bmax_bits);
    return;

drain:
    // a wait gave up: let this CTA's copies in flight land (bounded), then exit
    if (tid == 0) {
        if (streaming) {
            for (int64_t v = u; v < issued; ++v) mbar_wait_bounded(&H.bar[v & 1], (uint32_t)((v >> 1) & 1));
        } else {
            for (int64_t v = u; v < issued; ++v) mbar_wait_bounded(&H.bar[v], 0u);
        }
    }
    __syncthreads();
}

// Registers the integration and generation kernels of one (T, CPT, D, NB,
// CTAs per SM).
template <typename T, int CPT, int D_, int NB_, int MINB>
cudaError_t pass_launch_t(const Params& P, int mode, const PassArgs& A, int grid, size_t smem, cudaStream_t s)
{
    if (mode) k_pass<T, 1, CPT, D_, NB_, MINB><<<grid, PASS_THREADS, smem, s>>>(P, A);
    else k_pass<T, 0, CPT, D_, NB_, MINB><<<grid, PASS_THREADS, smem, s>>>(P, A);
    return cudaGetLastError();
}

template <typename T, int CPT, int D_, int NB_, int MINB = 2>
PassVariant make_variant()
{
    PassVariant v;
    v.fp32 = sizeof(T) == 4;
    v.cpt = CPT;
    v.D = D_;
    v.NB = NB_;
    v.minb = MINB;
    v.family = "k_pass";
    v.fn[0] = (const void*)k_pass<T, 0, CPT, D_, NB_, MINB>;
    v.fn[1] = (const void*)k_pass<T, 1, CPT, D_, NB_, MINB>;
    v.launch = &pass_launch_t<T, CPT, D_, NB_, MINB>;
    return v;
}

}  // namespace vamp

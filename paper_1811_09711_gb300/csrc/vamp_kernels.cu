// vamp_kernels.cu -- CUDA kernels of the multi-channel integrator's hot path.
//
//   k_begin_pass      integer call allocation N_c, prefix P_c (§3.4)
//   k_pass<T,0,CPT>   the sampling pass (§3.5 work order; Eqs. 15, 30, 31)
//   k_pass<T,1,CPT>   one generation batch: α-random channel, accept
//                     u w_max < w, ordered compaction (§2 Eq. 2, §3.5)
//   k_finish_pass     per-channel means/variances, pass result, combination
//   k_refine          VEGAS rebinning of every (channel, axis) row (Eqs. 14, 15)
//   k_update_alpha    channel-weight update (Eq. 25)
//   k_derive          lookup blocks: densities 1/(n Δx), cell tables, FP32 copies
//   k_gen_scan / k_gen_copy / k_gen_end   ordered output of a generation batch
//   k_eval<T>         per-call diagnostics for parity tests
//
// The pass kernel is persistent: each CTA owns a contiguous range of calls
// (integration) or a strided set of call chunks (generation), processed in
// batches of THREADS*CPT calls.  Per batch it streams the lookup blocks of
// all channels through shared memory in tiles, double-buffered with
// cp.async.bulk copies completing on mbarriers; every wait is bounded.
#include "vamp_device.cuh"
#include "vamp_internal.h"

namespace vamp {

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
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

// ---------------------------------------------------------------------------
// allocation (R6: N_c = max(N_min, floor(α_c N)) for α_c > 0)
// ---------------------------------------------------------------------------
__global__ void k_begin_pass(Params P, int64_t N)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t acc = 0;
        P.Pc[0] = 0;
        for (int c = 0; c < P.K; ++c) {
            int64_t nc = 0;
            if (P.alpha[c] > 0.0) {
                nc = (int64_t)floor(P.alpha[c] * (double)N);
                if (nc < P.n_min) nc = P.n_min;
            }
            P.Nc[c] = nc;
            acc += nc;
            P.Pc[c + 1] = acc;
        }
        P.sc->n_total = acc;
        P.sc->wmax_bits = 0ull;
    }
}

__device__ __forceinline__ int find_channel(const int64_t* Pc, int K, int64_t i)
{
    int lo = 0, hi = K - 1; // largest c with Pc[c] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (Pc[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// the pass kernel
// ---------------------------------------------------------------------------
struct SmemHead {
    uint64_t bar[2];
    int abort;
    int pad;
    double red[3][PASS_THREADS / 32];
    int wcnt[PASS_THREADS / 32];
    int woff[PASS_THREADS / 32];
    int round_total;
};

template <typename T, int MODE, int CPT>
__global__ void __launch_bounds__(PASS_THREADS, 2) k_pass(Params P, PassArgs A)
{
    extern __shared__ __align__(128) unsigned char smem[];
    SmemHead& H = *reinterpret_cast<SmemHead*>(smem);
    unsigned char* buf0 = smem + SMEM_HEAD;
    const BlkLayout& L = Prec<T>::lay(P);
    const int S = L.bytes;
    const size_t tile_bytes = (size_t)A.tile * S;
    double* Ds = reinterpret_cast<double*>(buf0 + (size_t)2 * A.tile * S);
    const int d = P.d, n = P.n, dn = d * n, K = P.K;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int B = PASS_THREADS * CPT;
    const unsigned char* lk = Prec<T>::lk(P);

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
        T p[CPT][DMAX], g[CPT], f[CPT], Aexp[CPT];
        bool skip[CPT], valid[CPT];
        int cq[CPT];
        uint32_t jp[CPT][4];
        uint32_t xacc[CPT];
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int64_t i = base + (int64_t)q * PASS_THREADS + tid;
            valid[q] = i < end;
            uint32_t X[DMAX + 4];
            call_words<DMAX + 4>(P, (uint32_t)(valid[q] ? i : base), A.field, MODE == 0 ? d : d + 2, X);
            int c;
            if (MODE == 0) {
                c = cseg;
                xacc[q] = 0u;
            } else {
                uint32_t xc = 0u, xa = 0u;
#pragma unroll
                for (int k = 0; k < DMAX + 4; ++k) {
                    if (k == d) xc = X[k];
                    if (k == d + 1) xa = X[k];
                }
                c = choose_channel(P, unif64(xc));
                xacc[q] = xa;
            }
            cq[q] = c;
            T x[DMAX];
            int jf[DMAX];
            T owngJ, Aq;
            forward_call<T>(P, c, X, x, p[q], jf, owngJ, Aq);
            Aexp[q] = Aq;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                uint32_t v = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) v |= (uint32_t)(jf[4 * w + b] & 0xff) << (8 * b);
                jp[q][w] = v;
            }
            g[q] = Prec<T>::alpha(P, c) * owngJ;
            f[q] = P.matching ? T(0) : integrand_peaks<T>(P, p[q], Aq);
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
            if (!H.abort) {
                const int cnt = min(A.tile, K - t * A.tile);
                for (int cl = 0; cl < cnt; ++cl) {
                    const int c2 = t * A.tile + cl;
                    const MapRec<T>& r = Prec<T>::ch(P)[c2];
                    const T a = Prec<T>::alpha(P, c2);
                    const bool lookups = (a != T(0)) && !(MODE == 0 && c2 == cseg);
#pragma unroll
                    for (int q = 0; q < CPT; ++q) skip[q] = (MODE == 1) && (cq[q] == c2);
                    const Blk<T> blk{buf0 + b * tile_bytes + (size_t)cl * S};
                    channel_body<T, CPT, false>(P, r, blk, a, lookups, P.matching != 0, p, Aexp, skip, g, f,
                                                nullptr);
                }
            }
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
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                if (!valid[q]) continue;
                double w = g[q] > T(0) ? (double)(f[q] / g[q]) : 0.0;
                if (!isfinite(w)) { bad = true; w = 0.0; }
                const double dv = w - sft;
                s1 += dv;
                s2 += dv * dv;
                wm = fmax(wm, w);
                const double w2 = w * w;
#pragma unroll
                for (int k = 0; k < DMAX; ++k)
                    if (k < d) atomicAdd(&Ds[k * n + ((jp[q][k >> 2] >> (8 * (k & 3))) & 0xff)], w2);
            }
            i0 = end;
            if (i0 >= seg_end) {
                // end of the segment: flush its sums and d-values
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
                s1 = s2 = 0.0;
                __syncthreads();
            }
        } else {
            const double wmax = P.sc->wmax_gen;
            int running = 0;
            const int64_t cbase = chunk * B;
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                double w = 0.0;
                bool acc = false;
                if (valid[q]) {
                    w = g[q] > T(0) ? (double)(f[q] / g[q]) : 0.0;
                    if (!isfinite(w)) { bad = true; w = 0.0; }
                    wm = fmax(wm, w);
                    acc = unif64(xacc[q]) * wmax < w;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, acc);
                if (lane == 0) H.wcnt[wid] = __popc(bal);
                __syncthreads();
                if (tid == 0) {
                    int s = 0;
                    for (int w2 = 0; w2 < PASS_THREADS / 32; ++w2) { H.woff[w2] = s; s += H.wcnt[w2]; }
                    H.round_total = s;
                }
                __syncthreads();
                if (acc) {
                    const int pos = running + H.woff[wid] + __popc(bal & ((1u << lane) - 1u));
                    const int64_t slot = cbase + pos;
                    unsigned char* rec = A.staging + slot * A.rec_bytes;
                    float* pf = reinterpret_cast<float*>(rec);
#pragma unroll
                    for (int k = 0; k < DMAX; ++k)
                        if (k < d) pf[k] = (float)p[q][k];
                    if (d & 1) pf[d] = 0.0f;
                    *reinterpret_cast<double*>(rec + A.rec_bytes - 8) = w;
                    A.callidx[slot] = (uint32_t)(base + (int64_t)q * PASS_THREADS + tid);
                }
                running += H.round_total;
                __syncthreads();
            }
            if (tid == 0) A.counts[chunk] = running;
            chunk += gridDim.x;
        }
    }

    // ---- CTA totals --------------------------------------------------------
    wm = warp_max(wm);
    if (lane == 0) H.red[2][wid] = wm;
    if (bad) atomicOr(&P.sc->err, ERR_NONFINITE);
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int q = 0; q < PASS_THREADS / 32; ++q) m = fmax(m, H.red[2][q]);
        unsigned long long* dst = MODE == 0 ? &P.sc->wmax_bits : &P.sc->gen_bmax_bits;
        atomicMax(dst, (unsigned long long)__double_as_longlong(m));
    }
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

// ---------------------------------------------------------------------------
// pass result (Eqs. 10, 11 per channel on shifted sums; Eq. 23; R8, R9)
// ---------------------------------------------------------------------------
__global__ void k_finish_pass(Params P, int combine)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Scalars* sc = P.sc;
    double I = 0.0, V = 0.0;
    for (int c = 0; c < P.K; ++c) {
        const int64_t nci = P.Nc[c];
        if (nci == 0) { P.Ic[c] = P.Vc[c] = P.Wc[c] = 0.0; continue; }
        const double Nc = (double)nci;
        const double m1 = P.csum[2 * c] / Nc, m2 = P.csum[2 * c + 1] / Nc;
        const double Ic = P.shift[c] + m1;
        double Vv = 0.0;
        if (nci > 1) Vv = (m2 - m1 * m1) * Nc / (Nc - 1.0);
        if (Vv < 0.0) Vv = 0.0;
        P.Ic[c] = Ic;
        P.Vc[c] = Vv;
        P.Wc[c] = (m2 - m1 * m1) + Ic * Ic;
    }
    for (int c = 0; c < P.K; ++c) {
        if (P.Nc[c] == 0) continue;
        I += P.alpha[c] * P.Ic[c];
        V += P.alpha[c] * P.alpha[c] * P.Vc[c] / (double)P.Nc[c];
    }
    for (int c = 0; c < P.K; ++c) P.shift[c] = P.Ic[c];
    const double wmax = __longlong_as_double((long long)sc->wmax_bits);
    sc->wmax_gen = wmax;
    const int h = sc->n_hist;
    if (h < 1024) {
        sc->hist_I[h] = I;
        sc->hist_V[h] = V;
        sc->hist_comb[h] = combine;
        sc->n_hist = h + 1;
    }
    // inverse-variance combination of the flagged passes
    int cnt = 0, nzero = 0;
    double zI = 0.0;
    for (int q = 0; q < sc->n_hist; ++q) {
        if (!sc->hist_comb[q]) continue;
        ++cnt;
        if (sc->hist_V[q] <= 0.0) { ++nzero; zI += sc->hist_I[q]; }
    }
    double cI = 0.0, cS = 0.0, chi = 0.0;
    if (cnt > 0 && nzero > 0) {
        cI = zI / nzero;
    } else if (cnt > 0) {
        double sw = 0.0, swi = 0.0;
        for (int q = 0; q < sc->n_hist; ++q) {
            if (!sc->hist_comb[q]) continue;
            sw += 1.0 / sc->hist_V[q];
            swi += sc->hist_I[q] / sc->hist_V[q];
        }
        cI = swi / sw;
        cS = sqrt(1.0 / sw);
        if (cnt > 1) {
            double ch = 0.0;
            for (int q = 0; q < sc->n_hist; ++q) {
                if (!sc->hist_comb[q]) continue;
                const double dI = sc->hist_I[q] - cI;
                ch += dI * dI / sc->hist_V[q];
            }
            chi = ch / (double)(cnt - 1);
        }
    }
    sc->res[0] = I;
    sc->res[1] = V;
    sc->res[2] = wmax;
    sc->res[3] = wmax > 0.0 ? I / wmax : 0.0;
    sc->res[4] = 0.0; // n_calls is taken from n_total on the host
    sc->res[5] = cI;
    sc->res[6] = cS;
    sc->res[7] = chi;
}

// ---------------------------------------------------------------------------
// lookup blocks of one grid row (Eq. 12 densities, FP32 copies, cell tables)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void derive_row_t(const Params& P, const BlkLayout& L, unsigned char* lk, int row,
                                             int lane, int nl)
{
    const int n = P.n, d = P.d;
    const int c = row / d, k = row % d;
    const double* e64 = P.edges64 + (size_t)row * (n + 1);
    unsigned char* blk = lk + (size_t)c * L.bytes;
    T* e = reinterpret_cast<T*>(blk) + k * L.Es;
    T* dnr = reinterpret_cast<T*>(blk + L.off_dens) + k * L.Dn;
    unsigned char* tb = blk + L.off_tab + k * L.Ts;
    for (int j = lane; j <= n; j += nl) {
        e[j] = (T)e64[j];
        if (j < n) dnr[j] = (T)(1.0 / ((double)n * (e64[j + 1] - e64[j])));
    }
    __syncwarp();
    // tb[q] = largest j in [0, n-1] with e[j] <= q/L, for q = 0..L
    const int Lc = 1 << L.lshift;
    int span = 0;
    for (int q = lane; q <= Lc; q += nl) {
        const T xq = (T)q / (T)Lc;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (e[mid] <= xq) lo = mid; else hi = mid - 1;
        }
        tb[q] = (unsigned char)lo;
    }
    __syncwarp();
    for (int q = lane; q < Lc; q += nl) span = max(span, (int)tb[q + 1] - (int)tb[q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) span = max(span, __shfl_xor_sync(0xffffffffu, span, o));
    if (lane == 0) blk[L.off_span + k] = (unsigned char)min(span, 255);
}

__device__ __forceinline__ void derive_row(const Params& P, int row, int lane)
{
    derive_row_t<double>(P, P.lay64, P.lk64, row, lane, 32);
    derive_row_t<float>(P, P.lay32, P.lk32, row, lane, 32);
}

__global__ void k_derive(Params P)
{
    const int rows = P.K * P.d;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int row = w; row < rows; row += nw) derive_row(P, row, lane);
    if (blockIdx.x == 0)
        for (int c = threadIdx.x; c < P.K; c += blockDim.x) P.alpha32[c] = (float)P.alpha[c];
}

// ---------------------------------------------------------------------------
// rebinning, one warp per (channel, axis) row (Eqs. 14, 15; R2-R4)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(REFINE_WARPS * 32) k_refine(Params P)
{
    extern __shared__ double rs[];
    const int n = P.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int row = blockIdx.x * REFINE_WARPS + wid;
    if (row >= P.K * P.d) return;
    double* Dj = rs + (size_t)wid * (4 * n + 2);
    double* m = Dj + n;
    double* C = m + n;          // n+1
    double* eo = C + n + 1;     // n+1
    const double* Din = P.D + (size_t)row * n;
    double* e = P.edges64 + (size_t)row * (n + 1);
    for (int j = lane; j < n; j += 32) Dj[j] = Din[j];
    for (int j = lane; j <= n; j += 32) eo[j] = e[j];
    __syncwarp();
    if (P.smooth && n >= 2) {
        for (int j = lane; j < n; j += 32) {
            double t;
            if (j == 0) t = (Dj[0] + Dj[1]) / 2.0;
            else if (j == n - 1) t = (Dj[n - 2] + Dj[n - 1]) / 2.0;
            else t = (Dj[j - 1] + Dj[j] + Dj[j + 1]) / 3.0;
            m[j] = t;
        }
        __syncwarp();
        for (int j = lane; j < n; j += 32) Dj[j] = m[j];
        __syncwarp();
    }
    for (int j = lane; j < n; j += 32) Dj[j] = sqrt(Dj[j]); // ω_j
    __syncwarp();
    double S = 0.0;
    if (lane == 0)
        for (int j = 0; j < n; ++j) S += Dj[j];
    S = __shfl_sync(0xffffffffu, S, 0);
    if (!(S > 0.0)) return;  // axis kept (R2); lookup blocks unchanged
    for (int j = lane; j < n; j += 32) {
        const double r = Dj[j] / S;
        double mj;
        if (r == 0.0) mj = 0.0;
        else if (fabs(r - 1.0) < 1e-12) mj = 1.0;
        else mj = pow((r - 1.0) / log(r), P.grid_alpha);
        m[j] = mj;
    }
    __syncwarp();
    double M = 0.0;
    if (lane == 0) {
        C[0] = 0.0;
        for (int j = 0; j < n; ++j) C[j + 1] = C[j] + m[j];
        M = C[n];
    }
    __syncwarp();
    M = __shfl_sync(0xffffffffu, M, 0);
    if (!(M > 0.0)) return;
    for (int i = lane; i <= n; i += 32) {
        double ne;
        if (i == 0) ne = 0.0;
        else if (i == n) ne = 1.0;
        else {
            const double t = (double)i * M / (double)n;
            int lo = 1, hi = n; // smallest j in [1, n] with C[j] >= t
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (C[mid] >= t) hi = mid; else lo = mid + 1;
            }
            const int j = lo;
            const double fr = (t - C[j - 1]) / m[j - 1];
            ne = __dadd_rn(eo[j - 1], __dmul_rn(fr, __dsub_rn(eo[j], eo[j - 1])));
        }
        e[i] = ne;
    }
    __syncwarp();
    derive_row(P, row, lane);
}

// ---------------------------------------------------------------------------
// channel weights (Eq. 25 with R5)
// ---------------------------------------------------------------------------
__global__ void k_update_alpha(Params P)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int K = P.K;
    double SU = 0.0, MU = 0.0;
    for (int c = 0; c < K; ++c) {
        const double om = P.omega_mode ? P.Wc[c] : P.Vc[c];
        if (P.alpha[c] > 0.0 && P.Nc[c] > 0 && om > 0.0) {
            SU += P.alpha[c] * pow(om, P.beta);
            MU += P.alpha[c];
        }
    }
    double tot = 0.0;
    // new weights go to Acum as scratch first
    for (int c = 0; c < K; ++c) {
        const double om = P.omega_mode ? P.Wc[c] : P.Vc[c];
        double a = P.alpha[c];
        if (a > 0.0 && P.Nc[c] > 0) {
            if (om > 0.0) a = P.alpha[c] * pow(om, P.beta) / SU * MU;
            else if (P.Ic[c] == 0.0) a = 0.0;
        }
        P.Acum[c] = a;
        tot += a;
    }
    if (tot > 0.0)
        for (int c = 0; c < K; ++c) P.alpha[c] = P.Acum[c] / tot;
    for (int c = 0; c < K; ++c) P.alpha32[c] = (float)P.alpha[c];
}

// ---------------------------------------------------------------------------
// generation bookkeeping
// ---------------------------------------------------------------------------
__global__ void k_gen_prepare(Params P)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc = 0.0;
    for (int c = 0; c < P.K; ++c) { acc += P.alpha[c]; P.Acum[c] = acc; }
    P.sc->gen_bmax_bits = 0ull;
}

// Exclusive prefix of the per-chunk counts, how many to take, calls used.
__global__ void k_gen_scan(Params P, PassArgs G, int64_t remaining)
{
    __shared__ long long part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nb = (int)G.nchunks;
    const int per = (nb + nt - 1) / nt;
    const int b0 = tid * per, b1 = min(nb, b0 + per);
    long long s = 0;
    for (int b = b0; b < b1; ++b) s += G.counts[b];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        long long a = 0;
        for (int q = 0; q < nt; ++q) { const long long v = part[q]; part[q] = a; a += v; }
        P.sc->gen_total = a;
        const long long take = a < remaining ? a : remaining;
        P.sc->gen_take = take;
        P.sc->gen_over = 0;
        P.sc->gen_used = G.batch;
    }
    __syncthreads();
    long long off = part[tid];
    const long long take = P.sc->gen_take;
    for (int b = b0; b < b1; ++b) {
        const long long cnt = G.counts[b];
        G.offsets[b] = off;
        // the chunk holding the last taken record decides the calls used
        if (take == remaining && take > 0 && off < take && take <= off + cnt) {
            const long long r = take - 1 - off;
            P.sc->gen_used = (long long)G.callidx[(int64_t)b * G.chunk + r] + 1;
        }
        off += cnt;
    }
}

__global__ void k_gen_copy(Params P, PassArgs G, unsigned char* out)
{
    const int b = blockIdx.x;
    const long long off = G.offsets[b], cnt = G.counts[b], take = P.sc->gen_take;
    if (off >= take) return;
    const long long ncopy = min(cnt, take - off);
    const int words = G.rec_bytes / 8;
    const unsigned long long* src =
        reinterpret_cast<const unsigned long long*>(G.staging + (int64_t)b * G.chunk * G.rec_bytes);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(out + off * G.rec_bytes);
    const double wmax = P.sc->wmax_gen;
    int over = 0;
    for (long long q = threadIdx.x; q < ncopy * words; q += blockDim.x) dst[q] = src[q];
    for (long long r = threadIdx.x; r < ncopy; r += blockDim.x) {
        const double w = *reinterpret_cast<const double*>(G.staging + ((int64_t)b * G.chunk + r) * G.rec_bytes +
                                                          (G.rec_bytes - 8));
        over += (w > wmax);
    }
    if (over) atomicAdd(reinterpret_cast<unsigned long long*>(&P.sc->gen_over), (unsigned long long)over);
}

__global__ void k_gen_end(Params P)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double bm = __longlong_as_double((long long)P.sc->gen_bmax_bits);
        if (bm > P.sc->wmax_gen) P.sc->wmax_gen = bm;
        P.sc->gen_bmax_bits = 0ull;
    }
}

// ---------------------------------------------------------------------------
// diagnostics: one call per thread, lookup blocks read from global memory
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_eval(Params P, EvalArgs A)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.count) return;
    const int d = P.d;
    const uint32_t call = A.call0 + (uint32_t)q;
    uint32_t X[DMAX + 4];
    int c;
    if (A.mode == 0) {
        call_words<DMAX + 4>(P, call, A.field, d, X);
        c = find_channel(P.Pc, P.K, (int64_t)call);
    } else {
        call_words<DMAX + 4>(P, call, A.field, d + 2, X);
        uint32_t xc = 0u;
        for (int k = 0; k < DMAX + 4; ++k)
            if (k == d) xc = X[k];
        c = choose_channel(P, unif64(xc));
    }
    T x[DMAX], p1[1][DMAX], g[1], f[1], Aq[1];
    bool skip[1];
    int jf[DMAX];
    T owngJ;
    forward_call<T>(P, c, X, x, p1[0], jf, owngJ, Aq[0]);
    g[0] = Prec<T>::alpha(P, c) * owngJ;
    f[0] = P.matching ? T(0) : integrand_peaks<T>(P, p1[0], Aq[0]);
    const BlkLayout& L = Prec<T>::lay(P);
    int* bins = A.bins + (size_t)q * P.K * d;
    for (int c2 = 0; c2 < P.K; ++c2) {
        const T a = Prec<T>::alpha(P, c2);
        const bool lookups = a != T(0) && c2 != c;
        skip[0] = false;
        const Blk<T> blk{Prec<T>::lk(P) + (size_t)c2 * L.bytes};
        channel_body<T, 1, true>(P, Prec<T>::ch(P)[c2], blk, a, lookups, P.matching != 0, p1, Aq, skip, g, f,
                                 bins + c2 * d);
        if (a == T(0))
            for (int k = 0; k < d; ++k) bins[c2 * d + k] = -1;
        else if (c2 == c)
            for (int k = 0; k < d; ++k) bins[c2 * d + k] = jf[k];
    }
    const T w = g[0] > T(0) ? f[0] / g[0] : T(0);
    for (int k = 0; k < d; ++k) {
        A.x[(size_t)q * d + k] = (double)x[k];
        A.p[(size_t)q * d + k] = (double)p1[0][k];
        A.jf[(size_t)q * d + k] = jf[k];
    }
    A.fgwc[4 * q + 0] = (double)f[0];
    A.fgwc[4 * q + 1] = (double)g[0];
    A.fgwc[4 * q + 2] = (double)w;
    A.fgwc[4 * q + 3] = (double)c;
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
cudaError_t launch_begin_pass(const Params& P, int64_t N, cudaStream_t s)
{
    k_begin_pass<<<1, 32, 0, s>>>(P, N);
    return cudaGetLastError();
}

template <typename T, int MODE>
static const void* pass_fn()
{
    return (const void*)k_pass<T, MODE, (sizeof(T) == 4 ? CPT32 : CPT64)>;
}

const void* pass_kernel(int fp32, int mode)
{
    if (fp32) return mode ? pass_fn<float, 1>() : pass_fn<float, 0>();
    return mode ? pass_fn<double, 1>() : pass_fn<double, 0>();
}

cudaError_t launch_pass(const Params& P, int fp32, int mode, const PassArgs& A, int grid, size_t smem,
                        cudaStream_t s)
{
    if (fp32) {
        if (mode) k_pass<float, 1, CPT32><<<grid, PASS_THREADS, smem, s>>>(P, A);
        else k_pass<float, 0, CPT32><<<grid, PASS_THREADS, smem, s>>>(P, A);
    } else {
        if (mode) k_pass<double, 1, CPT64><<<grid, PASS_THREADS, smem, s>>>(P, A);
        else k_pass<double, 0, CPT64><<<grid, PASS_THREADS, smem, s>>>(P, A);
    }
    return cudaGetLastError();
}

cudaError_t launch_finish_pass(const Params& P, int combine, cudaStream_t s)
{
    k_finish_pass<<<1, 32, 0, s>>>(P, combine);
    return cudaGetLastError();
}

cudaError_t launch_derive(const Params& P, cudaStream_t s)
{
    const int rows = P.K * P.d;
    const int blocks = min((rows + 3) / 4, 1024);
    k_derive<<<blocks, 128, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_refine(const Params& P, cudaStream_t s)
{
    const int rows = P.K * P.d;
    const int blocks = (rows + REFINE_WARPS - 1) / REFINE_WARPS;
    const size_t sm = (size_t)REFINE_WARPS * (4 * P.n + 2) * sizeof(double);
    k_refine<<<blocks, REFINE_WARPS * 32, sm, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_update_alpha(const Params& P, cudaStream_t s)
{
    k_update_alpha<<<1, 32, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_gen_prepare(const Params& P, cudaStream_t s)
{
    k_gen_prepare<<<1, 32, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_gen_finish(const Params& P, const PassArgs& G, int64_t remaining, unsigned char* out,
                              cudaStream_t s)
{
    k_gen_scan<<<1, 1024, 0, s>>>(P, G, remaining);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gen_copy<<<(unsigned)G.nchunks, 256, 0, s>>>(P, G, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gen_end<<<1, 32, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_eval(const Params& P, int fp32, const EvalArgs& A, cudaStream_t s)
{
    const int blocks = (A.count + 127) / 128;
    if (fp32) k_eval<float><<<blocks, 128, 0, s>>>(P, A);
    else k_eval<double><<<blocks, 128, 0, s>>>(P, A);
    return cudaGetLastError();
}

}  // namespace vamp

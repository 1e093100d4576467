// vamp_kernels.cu -- CUDA kernels of the multi-channel integrator's hot path.
//
//   k_begin_pass    integer call allocation N_c, prefix P_c (§3.4)
//   k_sample<T>     the sampling pass (§3.5 work order; Eqs. 15, 30, 31)
//   k_finish_pass   per-channel means/variances, pass result, combination
//   k_refine        VEGAS rebinning of every (channel, axis) row (Eqs. 14, 15)
//   k_update_alpha  channel-weight update (Eq. 25)
//   k_derive        bin densities 1/(n Δx) and FP32 copies of the grids
//   k_generate<T>   unweighted events: α-random channel, accept u w_max < w,
//                   ordered block compaction into staging (§2 Eq. 2, §3.5)
//   k_gen_scan / k_gen_copy / k_gen_end   ordered output of a batch
//   k_eval<T>       per-call diagnostics for parity tests
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <cfloat>

namespace vamp {

// ---------------------------------------------------------------------------
// block reductions
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
// sampling pass
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(SAMPLE_THREADS) k_sample(Params P, uint32_t iteration)
{
    extern __shared__ double smem[];
    double* Ds = smem;                       // [d][n] d-values of the current channel
    __shared__ double red_s1[SAMPLE_THREADS / 32], red_s2[SAMPLE_THREADS / 32],
        red_m[SAMPLE_THREADS / 32];
    const int d = P.d, n = P.n, dn = d * n;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t N = P.sc->n_total;
    const int64_t r0 = N * blockIdx.x / gridDim.x, r1 = N * (blockIdx.x + 1) / gridDim.x;
    double wm = 0.0;
    bool bad = false;
    int64_t i0 = r0;
    while (i0 < r1) {
        const int c = find_channel(P.Pc, P.K, i0);
        const int64_t seg_end = min(r1, P.Pc[c + 1]);
        for (int q = tid; q < dn; q += blockDim.x) Ds[q] = 0.0;
        __syncthreads();
        const double sft = P.shift[c];
        double s1 = 0.0, s2 = 0.0;
        for (int64_t i = i0 + tid; i < seg_end; i += blockDim.x) {
            uint32_t X[DMAX];
            call_words<DMAX>(P, (uint32_t)i, iteration, d, X);
            T x[DMAX], p[DMAX];
            int jf[DMAX];
            double w = (double)eval_call<T, false>(P, c, X, x, p, jf, nullptr, nullptr, nullptr);
            if (!isfinite(w)) { bad = true; w = 0.0; }
            const double dv = w - sft;
            s1 += dv;
            s2 += dv * dv;
            wm = fmax(wm, w);
            const double w2 = w * w;
#pragma unroll
            for (int k = 0; k < DMAX; ++k)
                if (k < d) atomicAdd(&Ds[k * n + jf[k]], w2);
        }
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if (lane == 0) { red_s1[wid] = s1; red_s2[wid] = s2; }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += red_s1[q]; b += red_s2[q]; }
            atomicAdd(&P.csum[2 * c], a);
            atomicAdd(&P.csum[2 * c + 1], b);
        }
        double* Dg = P.D + (size_t)c * dn;
        for (int q = tid; q < dn; q += blockDim.x) {
            const double v = Ds[q];
            if (v != 0.0) atomicAdd(&Dg[q], v);
        }
        __syncthreads();
        i0 = seg_end;
    }
    wm = warp_max(wm);
    if (lane == 0) red_m[wid] = wm;
    if (bad) atomicOr(&P.sc->err, ERR_NONFINITE);
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red_m[q]);
        atomicMax(&P.sc->wmax_bits, (unsigned long long)__double_as_longlong(m));
    }
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
// derived tables of one grid row: 1/(n Δx) (Eq. 12) and FP32 copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ void derive_row(const Params& P, int row, int lane, int nl)
{
    const int n = P.n;
    const double* e = P.edges64 + (size_t)row * (n + 1);
    double* dn = P.dens64 + (size_t)row * n;
    float* e32 = P.edges32 + (size_t)row * (n + 1);
    float* d32 = P.dens32 + (size_t)row * n;
    for (int j = lane; j <= n; j += nl) {
        e32[j] = (float)e[j];
        if (j < n) {
            const double v = 1.0 / ((double)n * (e[j + 1] - e[j]));
            dn[j] = v;
            d32[j] = (float)v;
        }
    }
}

__global__ void k_derive(Params P)
{
    const int rows = P.K * P.d;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) derive_row(P, row, threadIdx.x, blockDim.x);
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
    if (!(S > 0.0)) return;  // axis kept (R2); derived tables unchanged
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
    derive_row(P, row, lane, 32);
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
// generation
// ---------------------------------------------------------------------------
__global__ void k_gen_prepare(Params P)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc = 0.0;
    for (int c = 0; c < P.K; ++c) { acc += P.alpha[c]; P.Acum[c] = acc; }
    P.sc->gen_bmax_bits = 0ull;
}

template <typename T>
__device__ __forceinline__ void store_record(unsigned char* rec, int d, const T (&p)[DMAX], double w)
{
    float* pf = reinterpret_cast<float*>(rec);
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
        if (k < d) pf[k] = (float)p[k];
    if (d & 1) pf[d] = 0.0f;
    const int wo = ((4 * d + 7) & ~7);
    *reinterpret_cast<double*>(rec + wo) = w;
}

template <typename T>
__global__ void __launch_bounds__(GEN_THREADS) k_generate(Params P, GenArgs G)
{
    __shared__ int warp_cnt[GEN_THREADS / 32];
    __shared__ int warp_off[GEN_THREADS / 32];
    __shared__ double red_m[GEN_THREADS / 32];
    const int d = P.d;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * G.chunk;
    const double wmax = P.sc->wmax_gen;
    int running = 0;
    double bm = 0.0;
    bool bad = false;
    for (int64_t r = 0; r < G.chunk; r += GEN_THREADS) {
        const int64_t i = base + r + tid;
        bool acc = false;
        T x[DMAX], p[DMAX];
        double w = 0.0;
        if (i < G.batch) {
            uint32_t X[DMAX + 4];
            call_words<DMAX + 4>(P, (uint32_t)i, G.field, d + 2, X);
            uint32_t xc = 0u, xa = 0u; // words d and d+1 without dynamic indexing
#pragma unroll
            for (int k = 0; k < DMAX + 4; ++k) {
                if (k == d) xc = X[k];
                if (k == d + 1) xa = X[k];
            }
            const int c = choose_channel(P, unif64(xc));
            int jf[DMAX];
            w = (double)eval_call<T, false>(P, c, X, x, p, jf, nullptr, nullptr, nullptr);
            if (!isfinite(w)) { bad = true; w = 0.0; }
            bm = fmax(bm, w);
            acc = unif64(xa) * wmax < w;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, acc);
        if (lane == 0) warp_cnt[wid] = __popc(bal);
        __syncthreads();
        if (tid == 0) {
            int s = 0;
            for (int q = 0; q < GEN_THREADS / 32; ++q) { warp_off[q] = s; s += warp_cnt[q]; }
            warp_cnt[0] = s; // round total (read after the next barrier)
        }
        __syncthreads();
        if (acc) {
            const int pos = running + warp_off[wid] + __popc(bal & ((1u << lane) - 1u));
            const int64_t slot = base + pos;
            store_record<T>(G.staging + slot * G.rec_bytes, d, p, w);
            G.callidx[slot] = (uint32_t)i;
        }
        running += warp_cnt[0];
        __syncthreads();
    }
    if (tid == 0) G.counts[blockIdx.x] = running;
    bm = warp_max(bm);
    if (lane == 0) red_m[wid] = bm;
    if (bad) atomicOr(&P.sc->err, ERR_NONFINITE);
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int q = 0; q < GEN_THREADS / 32; ++q) m = fmax(m, red_m[q]);
        atomicMax(&P.sc->gen_bmax_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// Exclusive prefix of the per-block counts, how many to take, calls used.
__global__ void k_gen_scan(Params P, GenArgs G, int64_t remaining)
{
    __shared__ long long part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nb = G.nblocks;
    // each thread scans a contiguous slice
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
    const long long total = P.sc->gen_total;
    for (int b = b0; b < b1; ++b) {
        const long long cnt = G.counts[b];
        G.offsets[b] = off;
        // the block holding the last taken record decides the calls used
        if (take == remaining && take > 0 && off < take && take <= off + cnt) {
            const long long r = take - 1 - off;
            P.sc->gen_used = (long long)G.callidx[(int64_t)b * G.chunk + r] + 1;
        }
        off += cnt;
    }
    (void)total;
}

__global__ void k_gen_copy(Params P, GenArgs G, unsigned char* out)
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
// diagnostics
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
        c = choose_channel(P, unif64(X[d]));
    }
    T x[DMAX], p[DMAX], f, g;
    int jf[DMAX];
    const T w = eval_call<T, true>(P, c, X, x, p, jf, A.bins + (size_t)q * P.K * d, &f, &g);
    for (int k = 0; k < d; ++k) {
        A.x[(size_t)q * d + k] = (double)x[k];
        A.p[(size_t)q * d + k] = (double)p[k];
        A.jf[(size_t)q * d + k] = jf[k];
    }
    A.fgwc[4 * q + 0] = (double)f;
    A.fgwc[4 * q + 1] = (double)g;
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

template <typename T>
static cudaError_t launch_sample_t(const Params& P, uint32_t iteration, int grid, cudaStream_t s)
{
    const size_t sm = (size_t)P.d * P.n * sizeof(double);
    k_sample<T><<<grid, SAMPLE_THREADS, sm, s>>>(P, iteration);
    return cudaGetLastError();
}

cudaError_t launch_sample(const Params& P, int fp32, uint32_t iteration, int grid, cudaStream_t s)
{
    return fp32 ? launch_sample_t<float>(P, iteration, grid, s) : launch_sample_t<double>(P, iteration, grid, s);
}

cudaError_t sample_occupancy(int fp32, int d, int n, int* blocks_per_sm)
{
    const size_t sm = (size_t)d * n * sizeof(double);
    return fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sample<float>, SAMPLE_THREADS, sm)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sample<double>, SAMPLE_THREADS, sm);
}

cudaError_t launch_finish_pass(const Params& P, int combine, cudaStream_t s)
{
    k_finish_pass<<<1, 32, 0, s>>>(P, combine);
    return cudaGetLastError();
}

cudaError_t launch_derive(const Params& P, cudaStream_t s)
{
    const int rows = P.K * P.d;
    k_derive<<<rows < 1024 ? rows : 1024, 128, 0, s>>>(P);
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

cudaError_t launch_gen_batch(const Params& P, int fp32, const GenArgs& G, int64_t remaining, unsigned char* out,
                             cudaStream_t s)
{
    if (fp32) k_generate<float><<<G.nblocks, GEN_THREADS, 0, s>>>(P, G);
    else k_generate<double><<<G.nblocks, GEN_THREADS, 0, s>>>(P, G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gen_scan<<<1, 1024, 0, s>>>(P, G, remaining);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gen_copy<<<G.nblocks, 256, 0, s>>>(P, G, out);
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

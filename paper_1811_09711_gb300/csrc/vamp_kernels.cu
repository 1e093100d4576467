// vamp_kernels.cu -- the small kernels around the pass kernel (vamp_pass.cuh):
//
//   k_begin_pass      integer call allocation N_c, prefix P_c (§3.4); cells of a
//                     pseudo-stratified pass (§3.3)
//   k_strat_q         Σ over a channel's cells of the squared cell sums (§3.3)
//   k_finish_pass     per-channel means/variances, pass result, combination
//   k_pass_result     pass result into a caller's device array (asynchronous pass)
//   k_refine          VEGAS rebinning of every (channel, axis) row (Eqs. 14, 15),
//                     with the channel equivalences pooled in (§3.5)
//   k_update_alpha    channel-weight update (Eq. 25)
//   k_derive          lookup-block rows: densities 1/(n Δx), cell tables, FP32 copies
//   k_gen_prepare / k_gen_scan / k_gen_copy / k_gen_end   generation bookkeeping
//   k_eval<T>         per-call diagnostics for parity tests
//   k_batch_*         the same steps for every instance of a batch or server tick
#include "vamp_device.cuh"
#include "vamp_internal.h"

namespace vamp {

// ---------------------------------------------------------------------------
// allocation (R6: N_c = max(N_min, floor(α_c N)) for α_c > 0)
// ---------------------------------------------------------------------------
// Pseudo-stratified sampling (§3.3): the largest m in [1, 2^20] with
// 2 m^d <= N (exact integer search).
__device__ int64_t strat_cells_per_axis(int64_t N, int d)
{
    int64_t lo = 1, hi = 1 << 20;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        int64_t prod = 2;
        for (int k = 0; k < d && prod <= N; ++k) {
            if (prod > N / mid) { prod = N + 1; break; }
            prod *= mid;
        }
        if (prod <= N) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ void begin_pass_dev(const Params& P, int64_t N)
{
    {
        int64_t acc = 0, cells = 0;
        P.Pc[0] = 0;
        if (P.stratified) P.coff[0] = 0;
        for (int c = 0; c < P.K; ++c) {
            int64_t nc = 0;
            if (P.alpha[c] > 0.0) {
                nc = (int64_t)floor(P.alpha[c] * (double)N);
                if (nc < P.n_min) nc = P.n_min;
            }
            if (P.stratified) {
                // whole cells: n_r per axis, C = n_r^d cells, s = floor(N_c / C)
                int64_t m = 1, C = 1, s = nc;
                if (nc >= 2) {
                    m = strat_cells_per_axis(nc, P.d);
                    for (int k = 0; k < P.d; ++k) C *= m;
                    s = nc / C;
                }
                nc = s * C;
                P.nr[c] = m;
                P.spc[c] = s;
                cells += C;
                P.coff[c + 1] = cells;
            }
            P.Nc[c] = nc;
            acc += nc;
            P.Pc[c + 1] = acc;
        }
        P.sc->n_total = acc;
        P.sc->wmax_bits = 0ull;
    }
}

// Stratified passes: Q_c = Σ over the channel's cells of the squared cell
// sums, one 256-thread block per channel, fixed-order reduction (the same
// for a context and for an instance of a batch).
__device__ void strat_q_channel(const Params& P, int c)
{
    __shared__ double part[256];
    const int64_t a = P.coff[c], b = P.coff[c + 1];
    double s = 0.0;
    for (int64_t q = a + threadIdx.x; q < b; q += blockDim.x) {
        const double v = P.cellsum[q];
        s += v * v;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) P.Qc[c] = part[0];
}

__global__ void k_strat_q(Params P)
{
    strat_q_channel(P, blockIdx.x);
}

__global__ void k_begin_pass(Params P, int64_t N)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) begin_pass_dev(P, N);
}

// ---------------------------------------------------------------------------
// pass result (Eqs. 10, 11 per channel on shifted sums; Eq. 23; R8, R9)
// ---------------------------------------------------------------------------
// Called by every thread of one block: per-channel values in parallel, then
// thread 0 sums them in channel order (the order of the scalar form).
__device__ void finish_pass_dev(const Params& P, int combine)
{
    Scalars* sc = P.sc;
    for (int c = threadIdx.x; c < P.K; c += blockDim.x) {
        const int64_t nci = P.Nc[c];
        if (nci == 0) { P.Ic[c] = P.Vc[c] = P.Wc[c] = 0.0; P.shift[c] = 0.0; continue; }
        const double Nc = (double)nci;
        const double m1 = P.csum[2 * c] / Nc, m2 = P.csum[2 * c + 1] / Nc;
        const double Ic = P.shift[c] + m1;
        double Vv = 0.0;
        if (!P.stratified) {
            if (nci > 1) Vv = (m2 - m1 * m1) * Nc / (Nc - 1.0);
        } else if (P.spc[c] >= 2) {
            // mean over the channel's cells of the cells' sample variances
            const double s = (double)P.spc[c], C = (double)(P.coff[c + 1] - P.coff[c]);
            Vv = (P.csum[2 * c + 1] - P.Qc[c] / s) / (C * (s - 1.0));
        }
        if (Vv < 0.0) Vv = 0.0;
        P.Ic[c] = Ic;
        P.Vc[c] = Vv;
        P.Wc[c] = (m2 - m1 * m1) + Ic * Ic;
        P.shift[c] = Ic;  // R13: the next pass's sums are taken about this mean
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double I = 0.0, V = 0.0;
    for (int c = 0; c < P.K; ++c) {
        if (P.Nc[c] == 0) continue;
        I += P.alpha[c] * P.Ic[c];
        V += P.alpha[c] * P.alpha[c] * P.Vc[c] / (double)P.Nc[c];
    }
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

__global__ void k_finish_pass(Params P, int combine)
{
    finish_pass_dev(P, combine);
}

// Result of the last pass into a caller's device array (asynchronous form):
// integral, variance, w_max, efficiency, N', combined, its σ, χ²/dof, flags.
__global__ void k_pass_result(Params P, double* out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const Scalars* sc = P.sc;
    for (int q = 0; q < 8; ++q) out[q] = sc->res[q];
    out[4] = (double)sc->n_total;
    out[8] = (double)sc->err;
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
    unsigned char* r = lk + (size_t)c * L.bytes + L.H + (size_t)k * L.R;
    T* e = reinterpret_cast<T*>(r);
    T* dnr = reinterpret_cast<T*>(r + L.Es * sizeof(T));
    unsigned char* tb = r + (L.Es + L.Dn) * sizeof(T);
    // FP64 rows of mapped coordinates hold the images φ_c(ξ_j) of the edges
    // (clamped at 0, the forward map's formula): a bin of x = φ_c^{-1}(p) is
    // the bin whose image holds p, so the FP64 lookups compare p itself and
    // need no inverse map; the forward map reads the edges from the master
    // grid
    int kind = MAP_ID;
    const double* sp = nullptr;
    if (sizeof(T) == 8) {
        const ChanHdr<double>* h = reinterpret_cast<const ChanHdr<double>*>(lk + (size_t)c * L.bytes);
        if ((h->mask >> k) & 1u) {
            const int s = (int)((h->slotpack >> (4 * k)) & 0xFu);
            kind = (h->kinds >> (8 * s)) & 0xff;
            sp = h->sp[s];
        }
    }
    for (int j = lane; j <= n; j += nl) {
        double v = e64[j];
        if (kind == MAP_BW) {
            v = sp[SP_M] + sp[SP_G] * Prec<double>::tan_(sp[SP_A] * v - sp[SP_T0]);
        } else if (kind == MAP_POW) {
            const double v2 = v * v, v4 = v2 * v2;
            v = v4 * v;
            if (v < Prec<double>::tiny()) v = Prec<double>::tiny();
        }
        e[j] = (T)(v > 0.0 ? v : 0.0);
        const int jb = j < n ? j : n - 1;  // entry n repeats bin n-1
        dnr[j] = (T)(1.0 / ((double)n * (e64[jb + 1] - e64[jb])));
    }
    __syncwarp();
    // tb[q] = largest j in [0, n-1] with e[j] <= q/L, for q = 0..L
    const int Lc = 1 << L.lshift;
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
    int span = 0;
    for (int q = lane; q < Lc; q += nl) span = max(span, (int)tb[q + 1] - (int)tb[q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) span = max(span, __shfl_xor_sync(0xffffffffu, span, o));
    if (lane == 0) {
        tb[Lc + 1] = (unsigned char)min(span, 255);
        // this row's bit of the channel's slow-row mask (each row owns its bit)
        unsigned int* slow = reinterpret_cast<unsigned int*>(lk + (size_t)c * L.bytes + offsetof(ChanHdr<T>, slow));
        if (span > 1) atomicOr(slow, 1u << k);
        else atomicAnd(slow, ~(1u << k));
    }
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
// One warp rebins grid row `row` of P; ws = 4n+2 doubles of warp scratch.
__device__ void refine_row_dev(const Params& P, int row, int lane, double* ws)
{
    const int n = P.n;
    double* Dj = ws;
    double* m = Dj + n;
    double* C = m + n;          // n+1
    double* eo = C + n + 1;     // n+1
    const double* Din = P.D + (size_t)row * n;
    double* e = P.edges64 + (size_t)row * (n + 1);
    for (int j = lane; j < n; j += 32) Dj[j] = Din[j];
    if (P.eq_off) {
        // channel equivalences (§3.5): the pass's d-values of the equivalent
        // rows, added in list order (identity j, invert n-1-j, symmetric the
        // mean of both); an invariant axis takes unit weights
        const int q0 = P.eq_off[row], q1 = P.eq_off[row + 1];
        bool invariant = false;
        for (int q = q0; q < q1; ++q) {
            const int ent = P.eq_ent[q], kind = ent & 3;
            const double* src = P.D + (size_t)(ent >> 2) * n;
            if (kind == VAMP_EQ_INVARIANT) { invariant = true; continue; }
            for (int j = lane; j < n; j += 32) {
                double t;
                if (kind == VAMP_EQ_IDENTITY) t = src[j];
                else if (kind == VAMP_EQ_INVERT) t = src[n - 1 - j];
                else t = __dmul_rn(0.5, __dadd_rn(src[j], src[n - 1 - j]));
                Dj[j] = __dadd_rn(Dj[j], t);
            }
        }
        if (invariant)
            for (int j = lane; j < n; j += 32) Dj[j] = 1.0;
    }
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

__global__ void __launch_bounds__(REFINE_WARPS * 32) k_refine(Params P)
{
    extern __shared__ double rs[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int row = blockIdx.x * REFINE_WARPS + wid;
    if (row >= P.K * P.d) return;
    refine_row_dev(P, row, lane, rs + (size_t)wid * (4 * P.n + 2));
}

// ---------------------------------------------------------------------------
// channel weights (Eq. 25 with R5)
// ---------------------------------------------------------------------------
// Called by every thread of one block: the channel terms α_c ω_c^β in
// parallel (kept in Acum), the sums SU, MU and the normalisation by thread 0
// in channel order (the order of the scalar form).
__device__ void update_alpha_dev(const Params& P)
{
    __shared__ double red[2];
    const int K = P.K;
    auto omega = [&](int c) { return P.omega_mode ? P.Wc[c] : P.Vc[c]; };
    auto live = [&](int c) { return P.alpha[c] > 0.0 && P.Nc[c] > 0 && omega(c) > 0.0; };
    for (int c = threadIdx.x; c < K; c += blockDim.x)
        P.Acum[c] = live(c) ? P.alpha[c] * pow(omega(c), P.beta) : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double SU = 0.0, MU = 0.0;
        for (int c = 0; c < K; ++c) {
            if (live(c)) {
                SU += P.Acum[c];
                MU += P.alpha[c];
            }
        }
        red[0] = SU;
        red[1] = MU;
    }
    __syncthreads();
    const double SU = red[0], MU = red[1];
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        double a = P.alpha[c];
        if (a > 0.0 && P.Nc[c] > 0) {
            if (omega(c) > 0.0) a = P.Acum[c] / SU * MU;
            else if (P.Ic[c] == 0.0) a = 0.0;  // every call of the channel gave w = 0
        }
        P.Acum[c] = a;  // new weights, normalised below
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int c = 0; c < K; ++c) tot += P.Acum[c];
        red[0] = tot;
    }
    __syncthreads();
    const double tot = red[0];
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        if (tot > 0.0) P.alpha[c] = P.Acum[c] / tot;
        P.alpha32[c] = (float)P.alpha[c];
    }
}

__global__ void k_update_alpha(Params P)
{
    update_alpha_dev(P);
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
        over += (fabs(w) > wmax);
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
    using SH = Shape<T, 0, 0>;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.count) return;
    const SH sh(Prec<T>::lay(P), P.d, P.n);
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
    if (A.mode == 0 && P.stratified) {
        const uint32_t nr = (uint32_t)P.nr[c];
        uint32_t cell = (uint32_t)(((int64_t)call - P.Pc[c]) / P.spc[c]);
        uint32_t dig[DMAX];
        for (int k = 0; k < DMAX; ++k) {
            dig[k] = cell % nr;
            cell /= nr;
        }
        forward_call<T>(P, sh, c, X, x, p1[0], jf, owngJ, Aq[0], dig, nr);
    } else {
        forward_call<T>(P, sh, c, X, x, p1[0], jf, owngJ, Aq[0]);
    }
    g[0] = Prec<T>::alpha(P, c) * owngJ;
    f[0] = P.matching ? T(0) : integrand_peaks<T, DMAX>(P, d, p1[0], Aq[0]);
    int* bins = A.bins + (size_t)q * P.K * d;
    for (int c2 = 0; c2 < P.K; ++c2) {
        const T a = Prec<T>::alpha(P, c2);
        const bool lookups = a != T(0) && c2 != c;
        skip[0] = false;
        const unsigned char* blk = Prec<T>::lk(P) + (size_t)c2 * sh.bytes();
        channel_body<T, 1, true>(P, sh, blk, a, lookups, P.matching != 0, p1, Aq, skip, g, f, bins + c2 * d);
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
// many instances: the small steps of one iteration, one block (or warp) per
// instance (or grid row)
// ---------------------------------------------------------------------------
__global__ void k_batch_begin(MultiArgs M)
{
    const int i = blockIdx.x;
    if (i >= M.n_inst) return;
    const Params& P = M.inst[i];
    if (threadIdx.x == 0) begin_pass_dev(P, M.ncalls[i]);
    const size_t nd = (size_t)P.K * P.d * P.n;
    for (size_t q = threadIdx.x; q < nd; q += blockDim.x) P.D[q] = 0.0;
    for (int q = threadIdx.x; q < 2 * P.K; q += blockDim.x) P.csum[q] = 0.0;
    if (P.stratified) {
        // the cells of this pass (first cell of each channel set above)
        __syncthreads();
        const int64_t ncell = P.coff[P.K];
        for (int64_t q = threadIdx.x; q < ncell; q += blockDim.x) P.cellsum[q] = 0.0;
    }
}

// Stratified instances: Q_c per (instance, channel) pair, one block each.
__global__ void k_batch_strat_q(MultiArgs M)
{
    const int pair = blockIdx.x;
    int lo = 0, hi = M.n_inst - 1;  // instance of the pair
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (M.pair_off[mid] <= pair) lo = mid; else hi = mid - 1;
    }
    const Params& P = M.inst[lo];
    if (!P.stratified) return;
    strat_q_channel(P, pair - M.pair_off[lo]);
}

// Work items: every (instance, channel) pair with N_c calls gives
// ceil(N_c / item_calls) items; exclusive prefix over the pairs.
__global__ void k_batch_items(MultiArgs M)
{
    __shared__ long long part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (M.npairs + nt - 1) / nt;
    const int p0 = tid * per, p1 = min(M.npairs, p0 + per);
    auto items_of = [&](int pr) -> long long {
        int lo = 0, hi = M.n_inst - 1; // instance with pair_off[i] <= pr
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (M.pair_off[mid] <= pr) lo = mid; else hi = mid - 1;
        }
        const long long nc = M.inst[lo].Nc[pr - M.pair_off[lo]];
        return (nc + M.item_calls - 1) / M.item_calls;
    };
    long long s = 0;
    for (int pr = p0; pr < p1; ++pr) s += items_of(pr);
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        long long a = 0;
        for (int q = 0; q < nt; ++q) { const long long v = part[q]; part[q] = a; a += v; }
        M.ctl->total = a;
        M.ctl->next = 0;
        M.pair_prefix[M.npairs] = a;
    }
    __syncthreads();
    long long off = part[tid];
    for (int pr = p0; pr < p1; ++pr) {
        M.pair_prefix[pr] = off;
        off += items_of(pr);
    }
}

// one block per instance
__global__ void k_batch_finish(MultiArgs M)
{
    const int i = blockIdx.x;
    if (i >= M.n_inst) return;
    const Params& P = M.inst[i];
    finish_pass_dev(P, (int)M.iter[i] >= M.combine_from[i] ? 1 : 0);
    if (threadIdx.x != 0) return;
    double* r = M.results + (size_t)i * 9;
    for (int q = 0; q < 8; ++q) r[q] = P.sc->res[q];
    r[4] = (double)P.sc->n_total;
    r[8] = (double)P.sc->err;
}

__global__ void __launch_bounds__(REFINE_WARPS * 32) k_batch_refine(MultiArgs M)
{
    extern __shared__ double rs[];
    if (!(M.it->adapt & 1)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int row = blockIdx.x * REFINE_WARPS + wid;
    if (row >= M.nrows) return;
    int lo = 0, hi = M.n_inst - 1; // instance with row_off[i] <= row
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (M.row_off[mid] <= row) lo = mid; else hi = mid - 1;
    }
    refine_row_dev(M.inst[lo], row - M.row_off[lo], lane, rs + (size_t)wid * (4 * M.max_n + 2));
}

// one block per instance
__global__ void k_batch_alpha(MultiArgs M)
{
    if (!(M.it->adapt & 2)) return;
    const int i = blockIdx.x;
    if (i < M.n_inst) update_alpha_dev(M.inst[i]);
}

cudaError_t launch_batch_begin(const MultiArgs& M, cudaStream_t s)
{
    k_batch_begin<<<M.n_inst, 256, 0, s>>>(M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_batch_items<<<1, 1024, 0, s>>>(M);
    return cudaGetLastError();
}

cudaError_t launch_batch_after(const MultiArgs& M, cudaStream_t s)
{
    cudaError_t e;
    if (M.any_strat) {
        k_batch_strat_q<<<M.npairs, 256, 0, s>>>(M);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_batch_finish<<<M.n_inst, 64, 0, s>>>(M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int blocks = (M.nrows + REFINE_WARPS - 1) / REFINE_WARPS;
    k_batch_refine<<<blocks, REFINE_WARPS * 32, (size_t)REFINE_WARPS * (4 * M.max_n + 2) * sizeof(double), s>>>(M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_batch_alpha<<<M.n_inst, 64, 0, s>>>(M);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// self-test of the bounded wait: one CTA arms an mbarrier for a copy that is
// never issued, waits with the pass kernels' wait routine and a short limit,
// and records that it gave up (flag bit 0) and the cycles it waited
// ---------------------------------------------------------------------------
__global__ void k_wait_selftest(long long limit, unsigned int* flag, long long* cycles)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long t0 = clock64();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit);  // nothing completes phase 0
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(flag, ERR_TIMEOUT);
        *cycles = clock64() - t0;
    }
}

cudaError_t launch_wait_selftest(long long limit, unsigned int* flag, long long* cycles, cudaStream_t s)
{
    k_wait_selftest<<<1, 64, 0, s>>>(limit, flag, cycles);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
cudaError_t launch_begin_pass(const Params& P, int64_t N, cudaStream_t s)
{
    k_begin_pass<<<1, 32, 0, s>>>(P, N);
    return cudaGetLastError();
}

cudaError_t launch_strat_q(const Params& P, cudaStream_t s)
{
    k_strat_q<<<P.K, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_finish_pass(const Params& P, int combine, cudaStream_t s)
{
    k_finish_pass<<<1, 256, 0, s>>>(P, combine);
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

cudaError_t launch_pass_result(const Params& P, double* out, cudaStream_t s)
{
    k_pass_result<<<1, 32, 0, s>>>(P, out);
    return cudaGetLastError();
}

cudaError_t launch_update_alpha(const Params& P, cudaStream_t s)
{
    k_update_alpha<<<1, 256, 0, s>>>(P);
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

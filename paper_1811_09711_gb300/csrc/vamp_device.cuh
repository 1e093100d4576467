// vamp_device.cuh -- device-side building blocks of the sampling hot path.
//
// One call of the doubly adaptive multi-channel integrator (§3.5 work order):
//   r (Philox words) -> x_c = G_c^{-1}(r) on the selected channel's grid
//   -> p = φ_c(x_c) -> f(p) -> for every channel c': x_c' = φ_c'^{-1}(p),
//   bin lookup on grid c', g_c'(x_c') / φ'_c' -> g(p) (Eq. 30) -> w = f/g.
// Everything is templated on the evaluation type T: double (FP64 path) or
// float (FP32-eval path).  Sums are always FP64 (in the kernels).
//
// Grid data of one channel lives in one contiguous "lookup block" so that a
// tile of channels can be staged into shared memory with one bulk copy:
//   [edges  d rows x Es][densities d rows x Dn][cell tables d rows x Ts bytes][span d bytes]
// The cell table of a row splits [0,1) into L = 2^lshift equal cells and
// stores for cell q the bin containing q/L; a lookup then searches only the
// bins between two table entries (span = the widest such range of the row).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vamp {

constexpr int DMAX = 16;      // largest supported dimension
constexpr int MAXMAP = 4;     // mapped coordinates per channel / peak
constexpr int MAX_BINS = 256; // largest supported bins per axis (table entries are bytes)

enum : int { MAP_ID = 0, MAP_BW = 1, MAP_POW = 2 };
enum : unsigned { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

// One channel map or one integrand peak, with derived constants.
template <typename T>
struct MapRec {
    int32_t nmap;
    uint32_t mask;      // bit k: coordinate k is mapped
    uint64_t slotpack;  // 4 bits per coordinate: its slot
    int32_t kind[MAXMAP];
    T m[MAXMAP];        // Breit-Wigner mass
    T G[MAXMAP];        // Breit-Wigner width Γ
    T invG[MAXMAP];     // 1/Γ
    T A[MAXMAP];        // atan((1-m)/Γ) + atan(m/Γ)
    T GinvA[MAXMAP];    // Γ/A
    T invA[MAXMAP];     // 1/A
    T t0[MAXMAP];       // atan(m/Γ)
    T del[MAXMAP];      // power-law factor offset δ
    T invPowN[MAXMAP];  // 1 / (5((1+δ)^0.2 - δ^0.2))
    T wz;               // peak weight x Z^-(d - nmap) (Gaussian normalisation)
};

// Byte layout of one channel's lookup block for element type T.
struct BlkLayout {
    int Es;        // edges per row (>= n+1, padded)
    int Dn;        // densities per row (>= n, padded)
    int Ts;        // table bytes per row (>= L+1, padded)
    int lshift;    // L = 2^lshift cells per row
    int off_dens;  // byte offsets inside the block
    int off_tab;
    int off_span;
    int bytes;     // block size (multiple of 16)
};

// Device-resident scalars of one context.  The head (up to `n_hist`) is
// what the host copies back after a pass or a generation batch.
struct Scalars {
    int64_t n_total;                 // Σ N_c of the current pass
    unsigned long long wmax_bits;    // max weight of the pass (non-negative double bits)
    unsigned int err;                // ERR_* flags
    unsigned int pad0;
    double wmax_gen;                 // w_max used by generation
    double res[8];                   // pass result, vamp_pass_result order (n_calls slot unused)
    // generation batch bookkeeping
    unsigned long long gen_bmax_bits;
    long long gen_total;             // accepted in this batch
    long long gen_take;              // taken from this batch
    long long gen_used;              // calls consumed in this batch
    long long gen_over;              // overweights among taken
    // history of passes for the combination of iterations
    int32_t n_hist;
    int32_t pad1;
    double hist_I[1024];
    double hist_V[1024];
    int32_t hist_comb[1024];
};

// All pointers and sizes a kernel needs (passed by value).
struct Params {
    int d, K, n, P;
    int matching;          // peaks are the channels' maps (integrand fused into the channel loop)
    uint32_t key0, key1, request;
    int64_t n_min;
    double grid_alpha, beta;
    int smooth, omega_mode;
    // maps
    const MapRec<double>* ch64;
    const MapRec<float>* ch32;
    const MapRec<double>* pk64;
    const MapRec<float>* pk32;
    // Gaussian factor in log2 units: a_k = (p_k - centre)^2 * gk2
    double gcen, gk2;
    float gcen_f, gk2_f;
    // lookup blocks
    unsigned char* lk64;   // [K][lay64.bytes]
    unsigned char* lk32;   // [K][lay32.bytes]
    BlkLayout lay64, lay32;
    // state
    double* edges64;   // [K][d][n+1] FP64 master grid
    double* alpha;     // [K]
    float* alpha32;    // [K]
    double* shift;     // [K]
    double* Acum;      // [K] cumulative α for generation
    int64_t* Nc;       // [K]
    int64_t* Pc;       // [K+1]
    double* D;         // [K][d][n]
    double* csum;      // [K][2]: Σ (w - s_c), Σ (w - s_c)^2
    double* Ic;        // [K]
    double* Vc;        // [K]
    double* Wc;        // [K]
    Scalars* sc;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor round function with Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Words 0..nw-1 of one call (counter = call, block, field, request).
template <int NWMAX>
__device__ __forceinline__ void call_words(const Params& P, uint32_t call, uint32_t field, int nw,
                                           uint32_t (&X)[NWMAX])
{
#pragma unroll
    for (int b = 0; b < (NWMAX + 3) / 4; ++b) {
        if (4 * b < nw) {
            const uint4 o = philox4x32_10(make_uint4(call, (uint32_t)b, field, P.request), P.key0, P.key1);
            if (4 * b + 0 < NWMAX) X[4 * b + 0] = o.x;
            if (4 * b + 1 < NWMAX) X[4 * b + 1] = o.y;
            if (4 * b + 2 < NWMAX) X[4 * b + 2] = o.z;
            if (4 * b + 3 < NWMAX) X[4 * b + 3] = o.w;
        }
    }
}

// u = (X + 1/2) 2^-32 in (0, 1), exact in FP64.
__device__ __forceinline__ double unif64(uint32_t X) { return ((double)X + 0.5) * 0x1p-32; }

// ---------------------------------------------------------------------------
// Precision traits.
// ---------------------------------------------------------------------------
template <typename T> struct Prec;

template <> struct Prec<double> {
    static __device__ __forceinline__ const unsigned char* lk(const Params& P) { return P.lk64; }
    static __device__ __forceinline__ const BlkLayout& lay(const Params& P) { return P.lay64; }
    static __device__ __forceinline__ const MapRec<double>* ch(const Params& P) { return P.ch64; }
    static __device__ __forceinline__ const MapRec<double>* pk(const Params& P) { return P.pk64; }
    static __device__ __forceinline__ double alpha(const Params& P, int c) { return P.alpha[c]; }
    static __device__ __forceinline__ double gcen(const Params& P) { return P.gcen; }
    static __device__ __forceinline__ double gk2(const Params& P) { return P.gk2; }
    // in-bin fraction of the forward map: the exact 33-bit value
    static __device__ __forceinline__ double frac(uint64_t low33) { return (double)low33 * 0x1p-33; }
    // x = ξ_j + frac (ξ_{j+1} - ξ_j), rounded as two separate operations
    static __device__ __forceinline__ double lerp(double e0, double e1, double fr)
    {
        return __dadd_rn(e0, __dmul_rn(fr, __dsub_rn(e1, e0)));
    }
    static __device__ __forceinline__ double tan_(double v) { return tan(v); }
    static __device__ __forceinline__ double atan_(double v) { return atan(v); }
    static __device__ __forceinline__ double pow02(double v) { return pow(v, 0.2); }
    static __device__ __forceinline__ double powm08(double v) { return pow(v, -0.8); }
    static __device__ __forceinline__ double exp2_(double v) { return exp2(v); }
    static __device__ __forceinline__ double tiny() { return 2.2250738585072014e-308; }
    // e <= x for the non-negative edges: compare bit patterns (integer pipe)
    static __device__ __forceinline__ bool le(double e, double x)
    {
        return __double_as_longlong(e) <= __double_as_longlong(x);
    }
    // floor(x L) for x clamped to [0, 1): exact via round-toward-zero 1 + x
    static __device__ __forceinline__ int cell(double x, int lshift)
    {
        const double xc = fmin(fmax(x, 0.0), 0x1.fffffffffffffp-1);
        const double y = __dadd_rz(xc, 1.0);
        return (int)((unsigned long long)(__double_as_longlong(y) & 0xfffffffffffffll) >> (52 - lshift));
    }
};

template <> struct Prec<float> {
    static __device__ __forceinline__ const unsigned char* lk(const Params& P) { return P.lk32; }
    static __device__ __forceinline__ const BlkLayout& lay(const Params& P) { return P.lay32; }
    static __device__ __forceinline__ const MapRec<float>* ch(const Params& P) { return P.ch32; }
    static __device__ __forceinline__ const MapRec<float>* pk(const Params& P) { return P.pk32; }
    static __device__ __forceinline__ float alpha(const Params& P, int c) { return P.alpha32[c]; }
    static __device__ __forceinline__ float gcen(const Params& P) { return P.gcen_f; }
    static __device__ __forceinline__ float gk2(const Params& P) { return P.gk2_f; }
    // top 24 bits of the 33-bit fraction (exact conversion)
    static __device__ __forceinline__ float frac(uint64_t low33) { return (float)(uint32_t)(low33 >> 9) * 0x1p-24f; }
    static __device__ __forceinline__ float lerp(float e0, float e1, float fr) { return fmaf(fr, e1 - e0, e0); }
    static __device__ __forceinline__ float tan_(float v) { return tanf(v); }
    static __device__ __forceinline__ float atan_(float v) { return atanf(v); }
    static __device__ __forceinline__ float pow02(float v) { return exp2f(0.2f * __log2f(v)); }
    static __device__ __forceinline__ float powm08(float v) { return exp2f(-0.8f * __log2f(v)); }
    static __device__ __forceinline__ float exp2_(float v) { return exp2f(v); }
    static __device__ __forceinline__ float tiny() { return 1.17549435e-38f; }
    static __device__ __forceinline__ bool le(float e, float x) { return e <= x; }
    static __device__ __forceinline__ int cell(float x, int lshift)
    {
        const float xc = fminf(fmaxf(x, 0.0f), 0x1.fffffep-1f);
        const float y = __fadd_rz(xc, 1.0f);
        return (int)((__float_as_uint(y) & 0x7fffffu) >> (23 - lshift));
    }
};

__device__ __forceinline__ int slot_of(uint64_t slotpack, int k) { return (int)((slotpack >> (4 * k)) & 0xFu); }

// Views into a channel lookup block (global or shared memory).
template <typename T>
struct Blk {
    const unsigned char* b;
    __device__ __forceinline__ const T* e(const BlkLayout& L, int k) const
    {
        return reinterpret_cast<const T*>(b) + k * L.Es;
    }
    __device__ __forceinline__ const T* dn(const BlkLayout& L, int k) const
    {
        return reinterpret_cast<const T*>(b + L.off_dens) + k * L.Dn;
    }
    __device__ __forceinline__ const unsigned char* tb(const BlkLayout& L, int k) const
    {
        return b + L.off_tab + k * L.Ts;
    }
    __device__ __forceinline__ int span(const BlkLayout& L, int k) const { return b[L.off_span + k]; }
};

// Largest j in [0, n-1] with e[j] <= x (the oracle's bin rule), searching
// only between the table entries of x's cell.
template <typename T>
__device__ __forceinline__ int lookup(const T* e, const unsigned char* tb, int span, int lshift, T x)
{
    const int q = Prec<T>::cell(x, lshift);
    int j = tb[q];
    const int hi = tb[q + 1];
    if (span <= 1) {
        if (j < hi && Prec<T>::le(e[j + 1], x)) j += 1;
    } else {
        for (int s = 1 << (31 - __clz(span)); s > 0; s >>= 1) {
            const int t = j + s;
            if (t <= hi && Prec<T>::le(e[t], x)) j = t;
        }
    }
    return j;
}

// ---------------------------------------------------------------------------
// Forward map of the selected channel: r -> x_c -> p, g_c(x_c) / φ'_c(x_c),
// and the Gaussian exponent sum of p (log2 units).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void forward_call(const Params& P, int c, const uint32_t* X, T (&x)[DMAX],
                                             T (&p)[DMAX], int (&jf)[DMAX], T& own_gJ, T& asum_all)
{
    const int d = P.d, n = P.n;
    const BlkLayout& L = Prec<T>::lay(P);
    const Blk<T> blk{Prec<T>::lk(P) + (size_t)c * L.bytes};
    T g = T(1);
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            const uint64_t t = (2ull * X[k] + 1ull) * (uint64_t)n;
            const int j = (int)(t >> 33);
            const T fr = Prec<T>::frac(t & ((1ull << 33) - 1ull));
            const T* e = blk.e(L, k);
            x[k] = Prec<T>::lerp(__ldg(e + j), __ldg(e + j + 1), fr);
            jf[k] = j;
            g *= __ldg(blk.dn(L, k) + j);
        } else {
            x[k] = T(0);
            jf[k] = 0;
        }
    }
    const MapRec<T>& r = Prec<T>::ch(P)[c];
    const uint32_t mask = r.mask;
    T J = T(1), A = T(0);
    const T gc = Prec<T>::gcen(P), k2 = Prec<T>::gk2(P);
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        p[k] = x[k];
        if (k < d) {
            if ((mask >> k) & 1u) {
                const int s = slot_of(r.slotpack, k);
                if (r.kind[s] == MAP_BW) {
                    const T mass = r.m[s], G = r.G[s];
                    p[k] = mass + G * Prec<T>::tan_(r.A[s] * x[k] - r.t0[s]);
                    const T dp = p[k] - mass;
                    J *= r.GinvA[s] / (dp * dp + G * G);
                } else if (r.kind[s] == MAP_POW) {
                    const T x2 = x[k] * x[k], x4 = x2 * x2;
                    T pk = x4 * x[k];
                    if (pk < Prec<T>::tiny()) pk = Prec<T>::tiny();
                    p[k] = pk;
                    J *= T(1) / (T(5) * x4);
                }
            }
            const T u = p[k] - gc;
            A += u * u * k2;
        }
    }
    own_gJ = g * J;
    asum_all = A;
}

// ---------------------------------------------------------------------------
// One channel c' against CPT calls (the inner loop of Eq. 30, fused with
// the matching integrand peak when `with_f`):
//   g_q += α_c' g_c'(φ_c'^{-1}(p_q)) / φ'_c'   (unless skip_q)
//   f_q += wz_c' 2^-(A_q - Σ_mapped a_k) Π_mapped factor(p_k)
// REC records the bin indices of call 0 into bins[0..d-1].
// ---------------------------------------------------------------------------
template <typename T, int CPT, bool REC>
__device__ __forceinline__ void channel_body(const Params& P, const MapRec<T>& r, const Blk<T>& blk, T alpha_c,
                                             bool lookups, bool with_f, const T (&p)[CPT][DMAX],
                                             const T (&A)[CPT], const bool (&skip)[CPT], T (&g)[CPT],
                                             T (&f)[CPT], int* bins)
{
    const int d = P.d;
    const BlkLayout& L = Prec<T>::lay(P);
    const uint32_t mask = r.mask;
    const T gc = Prec<T>::gcen(P), k2 = Prec<T>::gk2(P);
    T J[CPT], F[CPT], gp[CPT], as[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) { J[q] = T(1); F[q] = T(1); gp[q] = T(1); as[q] = T(0); }
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            T xk[CPT];
#pragma unroll
            for (int q = 0; q < CPT; ++q) xk[q] = p[q][k];
            if ((mask >> k) & 1u) {
                const int s = slot_of(r.slotpack, k);
                if (r.kind[s] == MAP_BW) {
                    const T mass = r.m[s], G = r.G[s], invG = r.invG[s], GinvA = r.GinvA[s], invA = r.invA[s],
                            t0 = r.t0[s];
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        const T dp = p[q][k] - mass;
                        const T jfac = GinvA / (dp * dp + G * G);
                        J[q] *= jfac;
                        F[q] *= jfac;
                        xk[q] = (Prec<T>::atan_(dp * invG) + t0) * invA;
                        const T u = p[q][k] - gc;
                        as[q] += u * u * k2;
                    }
                } else if (r.kind[s] == MAP_POW) {
                    const T del = r.del[s], ipn = r.invPowN[s];
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        const T xx = Prec<T>::pow02(p[q][k]);
                        const T x2 = xx * xx;
                        J[q] *= T(1) / (T(5) * (x2 * x2));
                        xk[q] = xx;
                        if (with_f) F[q] *= Prec<T>::powm08(p[q][k] + del) * ipn;
                        const T u = p[q][k] - gc;
                        as[q] += u * u * k2;
                    }
                }
            }
            if (lookups) {
                const T* e = blk.e(L, k);
                const T* dn = blk.dn(L, k);
                const unsigned char* tb = blk.tb(L, k);
                const int sp = blk.span(L, k);
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int j = lookup<T>(e, tb, sp, L.lshift, xk[q]);
                    if (REC && q == 0) bins[k] = j;
                    gp[q] *= dn[j];
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        if (lookups && !skip[q]) g[q] += alpha_c * gp[q] * J[q];
        if (with_f) f[q] += r.wz * Prec<T>::exp2_(as[q] - A[q]) * F[q];
    }
}

// Integrand of a non-matching problem: loop over its own peaks.
template <typename T>
__device__ __forceinline__ T integrand_peaks(const Params& P, const T (&p)[DMAX], T A)
{
    const int d = P.d;
    const MapRec<T>* pks = Prec<T>::pk(P);
    const T gc = Prec<T>::gcen(P), k2 = Prec<T>::gk2(P);
    T f = T(0);
    for (int q = 0; q < P.P; ++q) {
        const MapRec<T>& r = pks[q];
        const uint32_t mask = r.mask;
        T v = T(1), as = T(0);
#pragma unroll
        for (int k = 0; k < DMAX; ++k) {
            if (k < d && ((mask >> k) & 1u)) {
                const int s = slot_of(r.slotpack, k);
                if (r.kind[s] == MAP_BW) {
                    const T dp = p[k] - r.m[s];
                    v *= r.GinvA[s] / (dp * dp + r.G[s] * r.G[s]);
                } else if (r.kind[s] == MAP_POW) {
                    v *= Prec<T>::powm08(p[k] + r.del[s]) * r.invPowN[s];
                }
                const T u = p[k] - gc;
                as += u * u * k2;
            }
        }
        f += r.wz * Prec<T>::exp2_(as - A) * v;
    }
    return f;
}

// Channel of a generation call: min{c : u A_K < A_c} on the cumulative α.
__device__ __forceinline__ int choose_channel(const Params& P, double u)
{
    const double tgt = u * P.Acum[P.K - 1];
    int lo = 0, hi = P.K - 1; // first c with tgt < A_c
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (tgt < P.Acum[mid]) hi = mid; else lo = mid + 1;
    }
    if (!(tgt < P.Acum[lo])) { // rounding: last live channel
        for (int c = P.K - 1; c >= 0; --c)
            if (P.alpha[c] > 0.0) return c;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Bulk-copy staging (cp.async.bulk + mbarrier), with bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One thread: expect `bytes` on bar and start the copy global -> shared.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of bar; gives up after ~2^31 SM cycles (about a
// second) and returns false, so that no wait can hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

}  // namespace vamp

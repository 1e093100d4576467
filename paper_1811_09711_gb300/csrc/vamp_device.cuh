// vamp_device.cuh -- device-side building blocks of the sampling hot path.
//
// One call of the doubly adaptive multi-channel integrator (§3.5 work order):
//   r (Philox words) -> x_c = G_c^{-1}(r) on the selected channel's grid
//   -> p = φ_c(x_c) -> f(p) -> for every channel c': x_c' = φ_c'^{-1}(p),
//   bin lookup on grid c', g_c'(x_c') / φ'_c' -> g(p) (Eq. 30) -> w = f/g.
// Everything here is templated on the evaluation type T: double (the FP64
// path) or float (the FP32-eval path).  Sums are always FP64 (in callers).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vamp {

constexpr int DMAX = 16;      // largest supported dimension
constexpr int MAXMAP = 4;     // mapped coordinates per channel / peak
constexpr int MAX_BINS = 256; // largest supported bins per axis

enum : int { MAP_ID = 0, MAP_BW = 1, MAP_POW = 2 };
enum : unsigned { ERR_NONFINITE = 1u, ERR_GEN_LIMIT = 2u };

// One channel map or one integrand peak, with its derived constants.
template <typename T>
struct MapRec {
    int32_t nmap;
    uint32_t mask;      // bit k: coordinate k is mapped
    uint64_t slotpack;  // 4 bits per coordinate: its slot
    int32_t kind[MAXMAP];
    T m[MAXMAP];        // Breit-Wigner mass
    T G[MAXMAP];        // Breit-Wigner width Γ
    T A[MAXMAP];        // atan((1-m)/Γ) + atan(m/Γ)
    T t0[MAXMAP];       // atan(m/Γ)
    T del[MAXMAP];      // power-law factor offset δ
    T powN[MAXMAP];     // 5((1+δ)^0.2 - δ^0.2)
    T weight;           // peak weight (peaks only)
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
    int top_step;          // highest power of two <= n-1 (0 if n == 1)
    uint32_t key0, key1, request;
    int64_t n_min;
    double grid_alpha, beta;
    int smooth, omega_mode;
    // maps
    const MapRec<double>* ch64;
    const MapRec<float>* ch32;
    const MapRec<double>* pk64;
    const MapRec<float>* pk32;
    int gauss_on;
    double gcen, gsig_inv, gZinv;
    float gcen_f, gsig_inv_f, gZinv_f;
    // state (FP64 master + FP32 copies)
    double* edges64;   // [K][d][n+1]
    double* dens64;    // [K][d][n]
    float* edges32;    // [K][d][n+1]
    float* dens32;     // [K][d][n]
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
// Precision traits: grid pointers and elementary functions.
// ---------------------------------------------------------------------------
template <typename T> struct Prec;

template <> struct Prec<double> {
    static __device__ __forceinline__ const double* edges(const Params& P) { return P.edges64; }
    static __device__ __forceinline__ const double* dens(const Params& P) { return P.dens64; }
    static __device__ __forceinline__ const MapRec<double>* ch(const Params& P) { return P.ch64; }
    static __device__ __forceinline__ const MapRec<double>* pk(const Params& P) { return P.pk64; }
    static __device__ __forceinline__ double alpha(const Params& P, int c) { return P.alpha[c]; }
    // in-bin fraction of the forward map: exact 33-bit value
    static __device__ __forceinline__ double frac(uint64_t low33) { return (double)low33 * 0x1p-33; }
    // x = ξ_j + frac (ξ_{j+1} - ξ_j) rounded as two separate operations
    static __device__ __forceinline__ double lerp(double e0, double e1, double fr)
    {
        return __dadd_rn(e0, __dmul_rn(fr, __dsub_rn(e1, e0)));
    }
    static __device__ __forceinline__ double tan_(double v) { return tan(v); }
    static __device__ __forceinline__ double atan_(double v) { return atan(v); }
    static __device__ __forceinline__ double pow02(double v) { return pow(v, 0.2); }
    static __device__ __forceinline__ double powm08(double v) { return pow(v, -0.8); }
    static __device__ __forceinline__ double exp_(double v) { return exp(v); }
    static __device__ __forceinline__ double tiny() { return 2.2250738585072014e-308; }
    static __device__ __forceinline__ double gcen(const Params& P) { return P.gcen; }
    static __device__ __forceinline__ double gsig_inv(const Params& P) { return P.gsig_inv; }
    static __device__ __forceinline__ double gZinv(const Params& P) { return P.gZinv; }
    // largest j in [0, n-1] with e[j] <= x; non-negative doubles compare as
    // their bit patterns, so the search runs on the integer pipe.
    static __device__ __forceinline__ int search(const double* e, int top, int nm1, double x)
    {
        const long long xb = __double_as_longlong(x);
        int j = 0;
        for (int step = top; step > 0; step >>= 1) {
            const int t = j + step;
            if (t <= nm1 && __double_as_longlong(__ldg(e + t)) <= xb) j = t;
        }
        return j;
    }
};

template <> struct Prec<float> {
    static __device__ __forceinline__ const float* edges(const Params& P) { return P.edges32; }
    static __device__ __forceinline__ const float* dens(const Params& P) { return P.dens32; }
    static __device__ __forceinline__ const MapRec<float>* ch(const Params& P) { return P.ch32; }
    static __device__ __forceinline__ const MapRec<float>* pk(const Params& P) { return P.pk32; }
    static __device__ __forceinline__ float alpha(const Params& P, int c) { return P.alpha32[c]; }
    // top 24 bits of the 33-bit fraction (exact conversion)
    static __device__ __forceinline__ float frac(uint64_t low33)
    {
        return (float)(uint32_t)(low33 >> 9) * 0x1p-24f;
    }
    static __device__ __forceinline__ float lerp(float e0, float e1, float fr) { return fmaf(fr, e1 - e0, e0); }
    static __device__ __forceinline__ float tan_(float v) { return tanf(v); }
    static __device__ __forceinline__ float atan_(float v) { return atanf(v); }
    static __device__ __forceinline__ float pow02(float v) { return powf(v, 0.2f); }
    static __device__ __forceinline__ float powm08(float v) { return powf(v, -0.8f); }
    static __device__ __forceinline__ float exp_(float v) { return expf(v); }
    static __device__ __forceinline__ float tiny() { return 1.17549435e-38f; }
    static __device__ __forceinline__ float gcen(const Params& P) { return P.gcen_f; }
    static __device__ __forceinline__ float gsig_inv(const Params& P) { return P.gsig_inv_f; }
    static __device__ __forceinline__ float gZinv(const Params& P) { return P.gZinv_f; }
    static __device__ __forceinline__ int search(const float* e, int top, int nm1, float x)
    {
        int j = 0;
        for (int step = top; step > 0; step >>= 1) {
            const int t = j + step;
            if (t <= nm1 && __ldg(e + t) <= x) j = t;
        }
        return j;
    }
};

__device__ __forceinline__ int slot_of(uint64_t slotpack, int k) { return (int)((slotpack >> (4 * k)) & 0xFu); }

// ---------------------------------------------------------------------------
// Synthetic integrand f(p) = Σ_q w_q Π_k (mapped ? factor : Gaussian).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T peak_factor(const MapRec<T>& r, int s, T pk)
{
    if (r.kind[s] == MAP_BW) {
        const T dp = pk - r.m[s], G = r.G[s];
        return G / (r.A[s] * (dp * dp + G * G));
    }
    if (r.kind[s] == MAP_POW) return Prec<T>::powm08(pk + r.del[s]) / r.powN[s];
    return T(1);
}

template <typename T>
__device__ __forceinline__ T integrand(const Params& P, const T (&p)[DMAX])
{
    const int d = P.d;
    T gk[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        gk[k] = T(1);
        if (k < d && P.gauss_on) {
            const T u = (p[k] - Prec<T>::gcen(P)) * Prec<T>::gsig_inv(P);
            gk[k] = Prec<T>::exp_(T(-0.5) * u * u) * Prec<T>::gZinv(P);
        }
    }
    const MapRec<T>* pks = Prec<T>::pk(P);
    T f = T(0);
    for (int q = 0; q < P.P; ++q) {
        const MapRec<T>& r = pks[q];
        const uint32_t mask = r.mask;
        T v = T(1);
#pragma unroll
        for (int k = 0; k < DMAX; ++k) {
            if (k < d) {
                if ((mask >> k) & 1u) v *= peak_factor(r, slot_of(r.slotpack, k), p[k]);
                else v *= gk[k];
            }
        }
        f += r.weight * v;
    }
    return f;
}

// ---------------------------------------------------------------------------
// Forward map of the selected channel: r -> x_c -> p, g_c(x_c), 1/φ'_c.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void forward_call(const Params& P, int c, const uint32_t* X, T (&x)[DMAX],
                                             T (&p)[DMAX], int (&jf)[DMAX], T& gc, T& jac)
{
    const int d = P.d, n = P.n;
    const T* E = Prec<T>::edges(P) + (size_t)c * d * (n + 1);
    const T* Dn = Prec<T>::dens(P) + (size_t)c * d * n;
    T g = T(1);
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            const uint64_t t = (2ull * X[k] + 1ull) * (uint64_t)n;
            const int j = (int)(t >> 33);
            const T fr = Prec<T>::frac(t & ((1ull << 33) - 1ull));
            const T e0 = __ldg(E + k * (n + 1) + j), e1 = __ldg(E + k * (n + 1) + j + 1);
            x[k] = Prec<T>::lerp(e0, e1, fr);
            jf[k] = j;
            g *= __ldg(Dn + k * n + j);
        } else {
            x[k] = T(0);
            jf[k] = 0;
        }
    }
    gc = g;
    const MapRec<T>& r = Prec<T>::ch(P)[c];
    T J = T(1);
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        p[k] = x[k];
        if (k < d && ((r.mask >> k) & 1u)) {
            const int s = slot_of(r.slotpack, k);
            if (r.kind[s] == MAP_BW) {
                const T mass = r.m[s], G = r.G[s], A = r.A[s];
                p[k] = mass + G * Prec<T>::tan_(A * x[k] - r.t0[s]);
                const T dp = p[k] - mass;
                J *= G / (A * (dp * dp + G * G));
            } else if (r.kind[s] == MAP_POW) {
                const T x2 = x[k] * x[k], x4 = x2 * x2;
                T pk = x4 * x[k];
                if (pk < Prec<T>::tiny()) pk = Prec<T>::tiny();
                p[k] = pk;
                J *= T(1) / (T(5) * x4);
            }
        }
    }
    jac = J;
}

// One channel's term α_c' g_c'(φ_c'^{-1}(p)) / φ'_c' of Eq. 30, optionally
// recording its bin indices.
template <typename T, bool REC>
__device__ __forceinline__ T channel_term(const Params& P, int cq, const T (&p)[DMAX], int* bins)
{
    const int d = P.d, n = P.n;
    const MapRec<T>& r = Prec<T>::ch(P)[cq];
    const T* E = Prec<T>::edges(P) + (size_t)cq * d * (n + 1);
    const T* Dn = Prec<T>::dens(P) + (size_t)cq * d * n;
    const uint32_t mask = r.mask;
    T J = T(1), g = T(1);
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            T xk = p[k];
            if ((mask >> k) & 1u) {
                const int s = slot_of(r.slotpack, k);
                if (r.kind[s] == MAP_BW) {
                    const T mass = r.m[s], G = r.G[s], A = r.A[s];
                    const T dp = p[k] - mass;
                    xk = (Prec<T>::atan_(dp / G) + r.t0[s]) / A;
                    J *= G / (A * (dp * dp + G * G));
                } else if (r.kind[s] == MAP_POW) {
                    xk = Prec<T>::pow02(p[k]);
                    const T x2 = xk * xk;
                    J *= T(1) / (T(5) * (x2 * x2));
                }
            }
            const int j = Prec<T>::search(E + k * (n + 1), P.top_step, n - 1, xk);
            if (REC) bins[k] = j;
            g *= __ldg(Dn + k * n + j);
        }
    }
    return Prec<T>::alpha(P, cq) * g * J;
}

// w = f(p) / g(p) for a call of channel c with words X (§3.5).
template <typename T, bool REC>
__device__ __forceinline__ T eval_call(const Params& P, int c, const uint32_t* X, T (&x)[DMAX], T (&p)[DMAX],
                                       int (&jf)[DMAX], int* bins, T* f_out, T* g_out)
{
    T gc, jac;
    forward_call<T>(P, c, X, x, p, jf, gc, jac);
    const T f = integrand<T>(P, p);
    T g = T(0);
    for (int cq = 0; cq < P.K; ++cq) {
        if (P.alpha[cq] == 0.0) {
            if (REC) for (int k = 0; k < P.d; ++k) bins[cq * P.d + k] = -1;
            continue;
        }
        T term;
        if (cq == c) {
            if (REC) for (int k = 0; k < P.d; ++k) bins[cq * P.d + k] = jf[k];
            term = Prec<T>::alpha(P, cq) * gc * jac;
        } else {
            term = channel_term<T, REC>(P, cq, p, REC ? bins + cq * P.d : nullptr);
        }
        g += term;
    }
    if (f_out) *f_out = f;
    if (g_out) *g_out = g;
    if (!(g > T(0))) return T(0);
    return f / g;
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

}  // namespace vamp

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
//   [header: map constants of the channel]
//   [row 0: edges (Es) | densities 1/(nΔx) (Dn) | cell table (Ts bytes)] [row 1] ...
// The cell table of a row splits [0,1) into L = 2^lshift equal cells and
// stores for cell q the bin containing q/L (byte L+1 holds the row's span:
// the most bins any cell overlaps), so a lookup starts next to its answer.
// Density entry n repeats entry n-1, so that a probe of edge ξ_n = 1 by a
// point at (or rounded past) 1 needs no bounds check: it lands on entry n
// with the last bin's density.  In the FP64 blocks the rows of mapped
// coordinates hold the images φ_c(ξ_j) of the edges (and their cell table
// is over p): the maps are increasing, so the bin of φ_c^{-1}(p) is the bin
// whose image holds p, found with no inverse map.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace vamp {

constexpr int DMAX = 16;      // largest supported dimension
constexpr int PASS_THREADS_DEV = 256;  // threads per pass CTA (PASS_THREADS of vamp_internal.h)
constexpr int MAXMAP = 4;     // mapped coordinates per channel / peak
constexpr int MAX_BINS = 256; // largest supported bins per axis (table entries are bytes)

enum : int { MAP_ID = 0, MAP_BW = 1, MAP_POW = 2 };
enum : unsigned { ERR_NONFINITE = 1u, ERR_TIMEOUT = 2u };

// Map constants of one channel or peak (used from global memory by the
// non-matching integrand path and by the host).
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

// Slot constants inside a lookup-block header.
enum : int { SP_M = 0, SP_G, SP_A, SP_G2, SP_INVG, SP_GINVA, SP_INVA, SP_T0, SP_DEL, SP_INVPOWN, SP_N };

// Header of a lookup block: what the channel loop needs about channel c'.
template <typename T>
struct ChanHdr {
    uint32_t mask;       // bit k: coordinate k is mapped
    uint32_t kinds;      // byte s: map kind of slot s
    uint64_t slotpack;   // 4 bits per coordinate: its slot
    T wz;                // matching peak: weight x Z^-(d - nmap)
    uint32_t slow;       // bit k: some cell of row k overlaps more than two bins (kept by the derive kernel)
    uint32_t pad[(16 - (sizeof(T) + 4) % 16) % 16 / 4];
    T sp[MAXMAP][SP_N];  // per slot: m, Γ, A, Γ², 1/Γ, Γ/A, 1/A, atan(m/Γ), δ, 1/powN
};
static_assert(sizeof(ChanHdr<float>) % 16 == 0 && sizeof(ChanHdr<double>) % 16 == 0, "header not 16-byte sized");

// Byte layout of one channel's lookup block for element type T.
struct BlkLayout {
    int H;         // header bytes
    int Es;        // edges per row (>= n+1, padded)
    int Dn;        // densities per row (>= n+1, padded; entry n repeats entry n-1)
    int Ts;        // table bytes per row (>= L+2, padded)
    int R;         // row stride in bytes
    int lshift;    // L = 2^lshift cells per row
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
    // maps (host order, for the non-matching integrand)
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
    // pseudo-stratified sampling (§3.3), when stratified != 0
    int stratified;
    int64_t* nr;       // [K] cells per r axis
    int64_t* spc;      // [K] calls per cell
    int64_t* coff;     // [K+1] first cell of each channel
    double* Qc;        // [K] Σ over the channel's cells of (Σ_cell (w - s_c))^2
    double* cellsum;   // [Σ cells] Σ_cell (w - s_c) of the pass (context-owned, grows)
    // channel equivalences (§3.5): the bin weights that rebin grid row r are
    // D[r] plus the terms eq_ent[eq_off[r] .. eq_off[r+1]) in list order, each
    // (source row << 2 | kind); null without equivalences
    int n_eq_ent;
    const int32_t* eq_off;   // [K*d + 1]
    const int32_t* eq_ent;   // [n_eq_ent]
    // interval tables of the FP32-eval union pass (null unless that kernel
    // is in use; rebuilt whenever the grids change): for coordinate k the
    // sorted distinct values U_k of every channel's edge images φ_c(ξ_{c,k,j})
    // (rounded up to FP32), a cell index over them, and for each interval
    // [U_k[u], U_k[u+1]) the bin densities of all channels (UNION_SLOTS wide)
    int uMax;          // row stride of uImg / uU / uD: K (n+1)
    float* uImg;       // [d][K][n+1] edge images per coordinate and channel
    float* uU;         // [d][uMax] sorted distinct images (first uNU[k] valid)
    int* uNU;          // [d]
    uint32_t* uC;      // [d][UNION_CELLS]: count of U_k <= q/L (low 16 bits), values inside the cell (high 16)
    float* uD;         // [d][uMax][UNION_SLOTS] densities of every channel on each interval
};

constexpr int UNION_SLOTS = 64;        // channels per density row of the union tables
constexpr int UNION_LCELLS = 16;       // log2 of the cells per coordinate of the union search
constexpr int UNION_CELLS = 1 << UNION_LCELLS;
constexpr int UNION_MAXV = 16384;      // largest K (n+1) the union tables take (16-bit indices, one sort block)

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
    static __device__ __forceinline__ const MapRec<double>* pk(const Params& P) { return P.pk64; }
    static __device__ __forceinline__ double alpha(const Params& P, int c) { return P.alpha[c]; }
    static __device__ __forceinline__ double gcen(const Params& P) { return P.gcen; }
    static __device__ __forceinline__ double gk2(const Params& P) { return P.gk2; }
    // in-bin fraction of the forward map: the exact 33-bit value
    static __device__ __forceinline__ double frac(uint64_t low33) { return (double)low33 * 0x1p-33; }
    // in-bin fraction of a stratified call: remainder over n_r 2^33, one
    // correctly rounded division
    static __device__ __forceinline__ double frac_div(uint64_t rem, uint64_t den)
    {
        return __ddiv_rn((double)rem, (double)den);
    }
    // x = ξ_j + frac (ξ_{j+1} - ξ_j), rounded as two separate operations
    static __device__ __forceinline__ double lerp(double e0, double e1, double fr)
    {
        return __dadd_rn(e0, __dmul_rn(fr, __dsub_rn(e1, e0)));
    }
    static __device__ __forceinline__ double tan_(double v) { return tan(v); }
    static __device__ __forceinline__ double atan_(double v) { return atan(v); }
    // v^(-1/5) for a normal v > 0 (Newton's method for the inverse fifth
    // root): with v = m 2^E, m in [1, 2), write -E = 5a + r (r in 0..4), so
    // v^(-1/5) = 2^a w^(-1/5) with w = m 2^-r in [1/16, 2).  The seed
    // 2^(-0.2 log2 w) comes from the FP32 special-function approximations
    // (relative error about 1e-7); two division-free Newton steps for
    // y^-5 = w, y <- y (6 - w y^5) / 5, each squaring the relative error,
    // bring it to a few units in the last place.
    static __device__ __forceinline__ double rinv5(double v)
    {
        const long long b = __double_as_longlong(v);
        const int ne = 1023 - (int)((b >> 52) & 0x7ff);  // -E
        const int a = ne >= 0 ? ne / 5 : -((4 - ne) / 5);
        const int r = ne - 5 * a;
        const double w = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | ((long long)(1023 - r) << 52));
        float s;
        float l;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"((float)w));  // w is normal
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(-0.2f * l));
        double y = (double)s;
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const double y2 = y * y, y4 = y2 * y2;
            y = y * fma(-w, y4 * y, 6.0) * 0.2;
        }
        return y * __longlong_as_double((long long)(1023 + a) << 52);  // times 2^a
    }
    // v^0.2 = v (v^(-1/5))^4
    static __device__ __forceinline__ double pow02(double v)
    {
        const double y = rinv5(v), y2 = y * y;
        return v * (y2 * y2);
    }
    // v^-0.8 = (v^(-1/5))^4
    static __device__ __forceinline__ double powm08(double v)
    {
        const double y = rinv5(v), y2 = y * y;
        return y2 * y2;
    }
    static __device__ __forceinline__ double exp2_(double v) { return exp2(v); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double tiny() { return 2.2250738585072014e-308; }
    // e <= x for the non-negative edges: compare bit patterns (integer pipe)
    static __device__ __forceinline__ bool le(double e, double x)
    {
        return __double_as_longlong(e) <= __double_as_longlong(x);
    }
    // floor(x L) for x clamped to [0, 1), from the bit pattern with integer
    // operations only (the FP64 pipe is the scarce one): x = m 2^(e-52) with
    // the 53-bit significand m, so floor(x 2^lshift) = m >> (52 - e - lshift)
    static __device__ __forceinline__ int cell(double x, int lshift)
    {
        const long long b = __double_as_longlong(x);
        if (b <= 0) return 0;                                    // x <= 0 (or -0)
        if (b >= 0x3FF0000000000000ll) return (1 << lshift) - 1; // x >= 1
        const int e = (int)(b >> 52) - 1023;                     // e <= -1
        const int sh = 52 - e - lshift;
        const unsigned long long m = (unsigned long long)(b & 0xFFFFFFFFFFFFFll) | (1ull << 52);
        return sh >= 64 ? 0 : (int)(m >> sh);
    }
};

template <> struct Prec<float> {
    static __device__ __forceinline__ const unsigned char* lk(const Params& P) { return P.lk32; }
    static __device__ __forceinline__ const BlkLayout& lay(const Params& P) { return P.lay32; }
    static __device__ __forceinline__ const MapRec<float>* pk(const Params& P) { return P.pk32; }
    static __device__ __forceinline__ float alpha(const Params& P, int c) { return P.alpha32[c]; }
    static __device__ __forceinline__ float gcen(const Params& P) { return P.gcen_f; }
    static __device__ __forceinline__ float gk2(const Params& P) { return P.gk2_f; }
    // top 24 bits of the 33-bit fraction (exact conversion)
    static __device__ __forceinline__ float frac(uint64_t low33) { return (float)(uint32_t)(low33 >> 9) * 0x1p-24f; }
    static __device__ __forceinline__ float frac_div(uint64_t rem, uint64_t den)
    {
        return (float)__ddiv_rn((double)rem, (double)den);
    }
    static __device__ __forceinline__ float lerp(float e0, float e1, float fr) { return fmaf(fr, e1 - e0, e0); }
    static __device__ __forceinline__ float tan_(float v) { return tanf(v); }
    static __device__ __forceinline__ float atan_(float v) { return atanf(v); }
    // 2^v by the ex2.approx instruction (relative error about 2^-22; flushes
    // results below the normal range to zero, where the factors it scales
    // are negligible)
    static __device__ __forceinline__ float ex2(float v)
    {
        float r;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
        return r;
    }
    // log2 v by the lg2.approx instruction, flush-to-zero form: the
    // arguments here are 0 or normal numbers (coordinates are sums and
    // products of uniform fractions and bin widths, and the power map
    // floors p at the smallest normal), on which it equals the form with
    // subnormal support and skips that form's rescaling steps
    static __device__ __forceinline__ float lg2(float v)
    {
        float r;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
        return r;
    }
    static __device__ __forceinline__ float pow02(float v) { return ex2(0.2f * lg2(v)); }
    static __device__ __forceinline__ float powm08(float v) { return ex2(-0.8f * lg2(v)); }
    static __device__ __forceinline__ float exp2_(float v) { return ex2(v); }
    // Jacobian factors of the FP32-eval form: a (1/b) by the div.approx
    // instruction (within 2 ulp for |b| in [2^-126, 2^126]), flush-to-zero
    // form: the denominators and quotients that occur here are normal
    static __device__ __forceinline__ float div(float a, float b)
    {
        float r;
        asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    }
    static __device__ __forceinline__ float tiny() { return 1.17549435e-38f; }
    static __device__ __forceinline__ bool le(float e, float x) { return e <= x; }
    // floor(x L) of x clamped to [0, 1], in [0, L]: x L + 2^23 rounded toward
    // zero is exact and its low mantissa bits are the integer part
    static __device__ __forceinline__ int cell(float x, int lshift)
    {
        const float y = __fmaf_rz(__saturatef(x), (float)(1 << lshift), 0x1p23f);
        return (int)(__float_as_uint(y) - 0x4B000000u);  // y - 2^23 (bit pattern of 2^23 is 0x4B000000)
    }
};

// ---------------------------------------------------------------------------
// Shape policy: D_, NB_ > 0 fix the dimension and the bins at compile time
// (all block offsets become constants); 0 means "read from the layout".
// With D_ = 0 the dimension is only known to lie in [DLO_, DMAX_]: loops run
// to DMAX_ and rows below DLO_ need no test (no branch in the unrolled loop).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ceil_log2(int v) { return v <= 1 ? 0 : 1 + ceil_log2((v + 1) / 2); }
__host__ __device__ constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }

template <typename T>
__host__ __device__ constexpr BlkLayout make_layout_c(int d, int n)
{
    const int per16 = 16 / (int)sizeof(T);
    const int es = round_up(n + 1, per16), dn = round_up(n + 1, per16);
    // about four cells per bin: on adapted grids nearly every row then has
    // no cell overlapping more than two bins (the single-probe lookup)
    const int ls = ceil_log2(n) + 2;
    const int ts = round_up((1 << ls) + 2, 16);
    const int h = (int)sizeof(ChanHdr<T>);
    const int r = (es + dn) * (int)sizeof(T) + ts;
    return BlkLayout{h, es, dn, ts, r, ls, h + d * r};
}

template <typename T, int D_, int NB_, int DMAX_ = DMAX, int DLO_ = 1>
struct Shape {
    static constexpr bool kD = D_ > 0, kN = NB_ > 0;
    static constexpr int DM = kD ? D_ : DMAX_;  // unrolled loop bound
    static constexpr int DLO = kD ? D_ : DLO_;  // rows below this always exist
    static constexpr int NBC = NB_;              // compile-time bins (0: runtime)
    // pseudo-stratified passes run only in the fully generic shape (the
    // specialised kernels are compiled without that code)
    static constexpr bool kStrat = !kD && !kN && DMAX_ == DMAX && DLO_ == 1;
    static constexpr BlkLayout C = make_layout_c<T>(kD ? D_ : 1, kN ? NB_ : 1);
    const BlkLayout L;
    const int d_rt, n_rt;
    __device__ __forceinline__ Shape(const BlkLayout& l, int d, int n) : L(l), d_rt(d), n_rt(n) {}
    __device__ __forceinline__ int d() const { return kD ? D_ : d_rt; }
    __device__ __forceinline__ bool has(int k) const { return k < DLO || k < d(); }
    __device__ __forceinline__ int n() const { return kN ? NB_ : n_rt; }
    __device__ __forceinline__ int H() const { return kN ? C.H : L.H; }
    __device__ __forceinline__ int R() const { return kN ? C.R : L.R; }
    __device__ __forceinline__ int dens_off() const { return kN ? C.Es * (int)sizeof(T) : L.Es * (int)sizeof(T); }
    __device__ __forceinline__ int tab_off() const { return kN ? (C.Es + C.Dn) * (int)sizeof(T) : (L.Es + L.Dn) * (int)sizeof(T); }
    __device__ __forceinline__ int lshift() const { return kN ? C.lshift : L.lshift; }
    __device__ __forceinline__ int bytes() const { return kN && kD ? C.bytes : L.bytes; }
    __device__ __forceinline__ const unsigned char* row(const unsigned char* blk, int k) const
    {
        return blk + H() + k * R();
    }
};

// Bin of x in a row whose cells overlap at most two bins: the cell's table
// entry, plus one if x reaches the next edge.
template <typename T, class SH>
__device__ __forceinline__ int lookup_fast(const SH& sh, const unsigned char* row, T x)
{
    const T* e = reinterpret_cast<const T*>(row);
    const int j = row[sh.tab_off() + Prec<T>::cell(x, sh.lshift())];
    return j + (Prec<T>::le(e[j + 1], x) ? 1 : 0);
}

// Largest j in [0, n-1] with e[j] <= x (the oracle's bin rule), starting at
// the table entry of x's cell.  A point at or past ξ_n = 1 may return n,
// whose density entry repeats bin n-1's.
template <typename T, class SH>
__device__ __forceinline__ int lookup(const SH& sh, const unsigned char* row, int span, T x)
{
    const T* e = reinterpret_cast<const T*>(row);
    const int q = Prec<T>::cell(x, sh.lshift());
    int j = row[sh.tab_off() + q];
    const int nm1 = sh.n() - 1;
    if (span <= 1) {
        j += Prec<T>::le(e[j + 1], x) ? 1 : 0;
    } else {
        for (int s = 1 << (31 - __clz(span)); s > 0; s >>= 1) {
            const int t = j + s;
            if (t <= nm1 && Prec<T>::le(e[t], x)) j = t;
        }
    }
    return j;
}

// ---------------------------------------------------------------------------
// Forward map of the selected channel (lookup block in global memory):
// r -> x_c -> p, the own term g_c(x_c)/φ'_c(x_c) and the Gaussian exponent
// sum of p (log2 units).
// ---------------------------------------------------------------------------
template <typename T, class SH>
__device__ __forceinline__ void forward_call(const Params& P, const SH& sh, int c, const uint32_t* X,
                                             T (&x)[SH::DM], T (&p)[SH::DM], int (&jf)[SH::DM], T& own_gJ,
                                             T& asum_all, const uint32_t* dig = nullptr, uint32_t nr = 1u)
{
    const int d = sh.d(), n = sh.n();
    const unsigned char* blk = Prec<T>::lk(P) + (size_t)c * sh.bytes();
    T g = T(1);
#pragma unroll
    for (int k = 0; k < SH::DM; ++k) {
        if (sh.has(k)) {
            int j;
            T fr;
            if (dig) {
                // stratified call: r_k = (a_k + u_k) / n_r, from the integer
                // (2^33 a_k + 2X + 1) n over n_r 2^33 (n_r = 1: the line below)
                const uint64_t den = (uint64_t)nr << 33;
                const uint64_t t = (((uint64_t)dig[k] << 33) + 2ull * X[k] + 1ull) * (uint64_t)n;
                const uint64_t jj = t / den;
                j = (int)jj;
                fr = Prec<T>::frac_div(t - jj * den, den);
            } else {
                const uint64_t t = (2ull * X[k] + 1ull) * (uint64_t)n;
                j = (int)(t >> 33);
                fr = Prec<T>::frac(t & ((1ull << 33) - 1ull));
            }
            const unsigned char* row = sh.row(blk, k);
            // the grid's edges: the FP32 block row, or the FP64 master grid
            // (whose values the FP64 block holds only for unmapped rows)
            const T* e = sizeof(T) == 8
                             ? reinterpret_cast<const T*>(P.edges64 + ((size_t)c * d + k) * (size_t)(n + 1))
                             : reinterpret_cast<const T*>(row);
            x[k] = Prec<T>::lerp(__ldg(e + j), __ldg(e + j + 1), fr);
            jf[k] = j;
            g *= __ldg(reinterpret_cast<const T*>(row + sh.dens_off()) + j);
        } else {
            x[k] = T(0);
            jf[k] = 0;
        }
    }
    const ChanHdr<T>* h = reinterpret_cast<const ChanHdr<T>*>(blk);
    const uint32_t mask = __ldg(&h->mask), kinds = __ldg(&h->kinds);
    const uint64_t slotpack = __ldg(&h->slotpack);
    T J = T(1), A = T(0);
    const T gc = Prec<T>::gcen(P), k2 = Prec<T>::gk2(P);
#pragma unroll
    for (int k = 0; k < SH::DM; ++k) {
        p[k] = x[k];
        if (sh.has(k)) {
            if ((mask >> k) & 1u) {
                const int s = (int)((slotpack >> (4 * k)) & 0xFu);
                const int kind = (kinds >> (8 * s)) & 0xff;
                const T* sp = h->sp[s];
                if (kind == MAP_BW) {
                    const T mass = __ldg(sp + SP_M), G = __ldg(sp + SP_G), A_ = __ldg(sp + SP_A);
                    p[k] = mass + G * Prec<T>::tan_(A_ * x[k] - __ldg(sp + SP_T0));
                    const T dp = p[k] - mass;
                    J *= Prec<T>::div(__ldg(sp + SP_GINVA), dp * dp + __ldg(sp + SP_G2));
                } else if (kind == MAP_POW) {
                    const T x2 = x[k] * x[k], x4 = x2 * x2;
                    T pk = x4 * x[k];
                    if (pk < Prec<T>::tiny()) pk = Prec<T>::tiny();
                    p[k] = pk;
                    J *= Prec<T>::div(T(1), T(5) * x4);
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
// One channel c' (block in shared or global memory) against CPT calls: the
// inner loop of Eq. 30, fused with the matching integrand peak when with_f:
//   g_q += α_c' g_c'(φ_c'^{-1}(p_q)) / φ'_c'   (lookups and not skip_q)
//   f_q += wz_c' 2^-(A_q - Σ_mapped a_k) Π_mapped factor(p_k)
// REC records the bin indices of call 0 into bins[0..d-1].
// ---------------------------------------------------------------------------
// Rows of one channel against CPT calls: bin densities (gp), Jacobians of the
// mapped coordinates (J), matching-peak factors (F) and Gaussian exponents of
// the mapped coordinates (as).  FAST: every row's cells overlap at most two
// bins, so one edge probe settles each bin and the unrolled row loop has no
// branch other than the mapped-coordinate test; otherwise rows are tested
// one by one and only the spanning ones search.
// pw (FP64 pass kernel, else null): this thread's 0.2 p_k^(-4/5) per call q
// and coordinate k at pw[(q DM + k) PASS_THREADS], computed once per call,
// the power-law Jacobian of every channel that maps k.
template <typename T, int CPT, bool REC, bool FAST, class SH>
__device__ __forceinline__ void channel_rows(const Params& P, const SH& sh, const unsigned char* blk, bool with_f,
                                             const T (&p)[CPT][SH::DM], T (&J)[CPT], T (&F)[CPT], T (&gp)[CPT],
                                             T (&as)[CPT], int* bins, const T* pw)
{
    const int d = sh.d();
    const ChanHdr<T>& h = *reinterpret_cast<const ChanHdr<T>*>(blk);
    const uint32_t mask = h.mask, kinds = h.kinds, slow = h.slow;
    const uint64_t slotpack = h.slotpack;
    const T gc = Prec<T>::gcen(P), k2 = Prec<T>::gk2(P);
    // FP64: the Breit-Wigner Jacobians Γ/(A((p-m)² + Γ²)) of the channel as
    // one quotient of the products of numerators and denominators (one FP64
    // division per channel instead of one per mapped coordinate; each
    // denominator is at least Γ², so the product of four stays normal)
    T bw_num = T(1), bw_den[CPT];
    bool any_bw = false;
#pragma unroll
    for (int q = 0; q < CPT; ++q) bw_den[q] = T(1);
#pragma unroll
    for (int k = 0; k < SH::DM; ++k) {
        if (sh.has(k)) {
            T xk[CPT];
#pragma unroll
            for (int q = 0; q < CPT; ++q) xk[q] = p[q][k];
            if ((mask >> k) & 1u) {
                const int s = (int)((slotpack >> (4 * k)) & 0xFu);
                const int kind = (kinds >> (8 * s)) & 0xff;
                const T* sp = h.sp[s];
                if (kind == MAP_BW) {
                    const T mass = sp[SP_M], G2 = sp[SP_G2], invG = sp[SP_INVG], GinvA = sp[SP_GINVA],
                            invA = sp[SP_INVA], t0 = sp[SP_T0];
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        const T dp = p[q][k] - mass;
                        if constexpr (sizeof(T) == 8) {
                            // FP64 rows of mapped coordinates hold the images of
                            // the edges: the lookup compares p itself
                            bw_den[q] *= dp * dp + G2;
                        } else {
                            const T jfac = Prec<T>::div(GinvA, dp * dp + G2);
                            J[q] *= jfac;
                            F[q] *= jfac;
                            xk[q] = (Prec<T>::atan_(dp * invG) + t0) * invA;
                        }
                        const T u = p[q][k] - gc;
                        as[q] += u * u * k2;
                    }
                    if constexpr (sizeof(T) == 8) {
                        bw_num *= GinvA;
                        any_bw = true;
                    }
                } else if (kind == MAP_POW) {
                    const T del = sp[SP_DEL], ipn = sp[SP_INVPOWN];
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        if constexpr (sizeof(T) == 8) {
                            // 1/φ' = 1/(5 x^4) = y^4 / 5 with x = p^0.2 and
                            // y = p^(-1/5): no division, no pow (the lookup
                            // compares p with the edge images)
                            if (pw) {
                                J[q] *= pw[(q * SH::DM + k) * PASS_THREADS_DEV];
                            } else {
                                const T y = Prec<T>::rinv5(p[q][k]), y2 = y * y, y4 = y2 * y2;
                                J[q] *= T(0.2) * y4;
                            }
                        } else {
                            const T xx = Prec<T>::pow02(p[q][k]);
                            const T x2 = xx * xx;
                            J[q] *= Prec<T>::div(T(1), T(5) * (x2 * x2));
                            xk[q] = xx;
                        }
                        if (with_f) F[q] *= Prec<T>::powm08(p[q][k] + del) * ipn;
                        const T u = p[q][k] - gc;
                        as[q] += u * u * k2;
                    }
                }
            }
            // every channel's rows are probed; the terms of the own channel
            // and of switched-off channels are dropped by the caller
            const unsigned char* row = sh.row(blk, k);
            const T* dn = reinterpret_cast<const T*>(row + sh.dens_off());
            if (FAST) {
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int j = lookup_fast<T>(sh, row, xk[q]);
                    if (REC && q == 0) bins[k] = min(j, sh.n() - 1);
                    gp[q] *= dn[j];
                }
            } else if (!((slow >> k) & 1u)) {
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int j = lookup_fast<T>(sh, row, xk[q]);
                    if (REC && q == 0) bins[k] = min(j, sh.n() - 1);
                    gp[q] *= dn[j];
                }
            } else {
                const int sp = row[sh.tab_off() + (1 << sh.lshift()) + 1];
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int j = lookup<T>(sh, row, sp, xk[q]);
                    if (REC && q == 0) bins[k] = min(j, sh.n() - 1);
                    gp[q] *= dn[j];
                }
            }
        }
    }
    if constexpr (sizeof(T) == 8) {
        if (any_bw) {
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const T jb = Prec<T>::div(bw_num, bw_den[q]);
                J[q] *= jb;
                F[q] *= jb;
            }
        }
    }
}

template <typename T, int CPT, bool REC, class SH>
__device__ __forceinline__ void channel_body(const Params& P, const SH& sh, const unsigned char* blk, T alpha_c,
                                             bool lookups, bool with_f, const T (&p)[CPT][SH::DM],
                                             const T (&A)[CPT], const bool (&skip)[CPT], T (&g)[CPT],
                                             T (&f)[CPT], int* bins, const T* pw = nullptr)
{
    const ChanHdr<T>& h = *reinterpret_cast<const ChanHdr<T>*>(blk);
    T J[CPT], F[CPT], gp[CPT], as[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) { J[q] = T(1); F[q] = T(1); gp[q] = T(1); as[q] = T(0); }
    if (h.slow == 0u) channel_rows<T, CPT, REC, true>(P, sh, blk, with_f, p, J, F, gp, as, bins, pw);
    else channel_rows<T, CPT, REC, false>(P, sh, blk, with_f, p, J, F, gp, as, bins, pw);
    const T wz = h.wz;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        if (lookups && !skip[q]) g[q] += alpha_c * gp[q] * J[q];
        if (with_f) f[q] += wz * Prec<T>::exp2_(as[q] - A[q]) * F[q];
    }
}

// Integrand of a non-matching problem: loop over its own peaks.
template <typename T, int DM>
__device__ __forceinline__ T integrand_peaks(const Params& P, int d, const T (&p)[DM], T A)
{
    const MapRec<T>* pks = Prec<T>::pk(P);
    const T gc = Prec<T>::gcen(P), k2 = Prec<T>::gk2(P);
    T f = T(0);
    for (int q = 0; q < P.P; ++q) {
        const MapRec<T>& r = pks[q];
        const uint32_t mask = r.mask;
        T v = T(1), as = T(0);
#pragma unroll
        for (int k = 0; k < DM; ++k) {
            if (k < d && ((mask >> k) & 1u)) {
                const int s = (int)((r.slotpack >> (4 * k)) & 0xFu);
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

// Waits for phase `parity` of bar; gives up after `limit` SM cycles (by
// default 2^31, about a second) and returns false, so that no wait can hang
// the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = 1ll << 31)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

}  // namespace vamp

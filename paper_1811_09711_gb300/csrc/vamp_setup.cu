// vamp_setup.cu -- host-side setup shared by vamp_create and the
// allocation-free entry point: validation of a vamp_config, derived
// constants of the maps and the Gaussian factor, lookup-block layout and
// headers, placement of the per-problem arrays, pass-kernel variants.
#include "vamp_device.cuh"
#include "vamp_internal.h"

#include <cmath>
#include <cstring>
#include <mutex>

namespace vamp {

namespace {

bool check_maps(const vamp_map_desc* m, int cnt, int d, std::string& why)
{
    for (int q = 0; q < cnt; ++q) {
        const vamp_map_desc& r = m[q];
        if (r.n_mapped < 0 || r.n_mapped > MAXMAP) { why = "n_mapped out of range"; return false; }
        unsigned seen = 0;
        for (int s = 0; s < r.n_mapped; ++s) {
            const int k = r.coord[s];
            if (k < 0 || k >= d) { why = "mapped coordinate out of range"; return false; }
            if (seen & (1u << k)) { why = "coordinate mapped twice"; return false; }
            seen |= 1u << k;
            if (r.kind[s] == VAMP_MAP_BW) {
                if (!(r.b[s] > 0.0) || !std::isfinite(r.a[s]) || !std::isfinite(r.b[s])) {
                    why = "Breit-Wigner width must be > 0";
                    return false;
                }
            } else if (r.kind[s] == VAMP_MAP_POW) {
                if (!(r.b[s] >= 0.0) || !std::isfinite(r.b[s])) { why = "power-law delta must be >= 0"; return false; }
            } else if (r.kind[s] != VAMP_MAP_ID) {
                why = "unknown map kind";
                return false;
            }
        }
    }
    return true;
}

bool same_maps(const vamp_map_desc& a, const vamp_map_desc& b)
{
    if (a.n_mapped != b.n_mapped) return false;
    for (int s = 0; s < a.n_mapped; ++s)
        if (a.coord[s] != b.coord[s] || a.kind[s] != b.kind[s] || a.a[s] != b.a[s] || a.b[s] != b.b[s])
            return false;
    return true;
}

// Breit-Wigner constants: A = ∫_0^1 Γ/((p-m)²+Γ²) dp, t0 = atan(m/Γ);
// power law: 1 / ∫_0^1 (p+δ)^-0.8 dp.
double bw_A(double m, double G) { return std::atan((1.0 - m) / G) + std::atan(m / G); }
double pow_invN(double del) { return 1.0 / (5.0 * (std::pow(1.0 + del, 0.2) - std::pow(del, 0.2))); }

template <typename T>
MapRec<T> make_rec(const vamp_map_desc& r, double weight, double zinv, int d)
{
    MapRec<T> o;
    std::memset(&o, 0, sizeof o);
    o.nmap = r.n_mapped;
    o.wz = (T)(weight * std::pow(zinv, (double)(d - r.n_mapped)));
    for (int s = 0; s < r.n_mapped; ++s) {
        const int k = r.coord[s];
        o.mask |= 1u << k;
        o.slotpack |= (uint64_t)s << (4 * k);
        o.kind[s] = r.kind[s];
        if (r.kind[s] == VAMP_MAP_BW) {
            const double m = r.a[s], G = r.b[s], A = bw_A(m, G);
            o.m[s] = (T)m;
            o.G[s] = (T)G;
            o.invG[s] = (T)(1.0 / G);
            o.A[s] = (T)A;
            o.GinvA[s] = (T)(G / A);
            o.invA[s] = (T)(1.0 / A);
            o.t0[s] = (T)std::atan(m / G);
        } else if (r.kind[s] == VAMP_MAP_POW) {
            o.del[s] = (T)r.b[s];
            o.invPowN[s] = (T)pow_invN(r.b[s]);
        }
    }
    return o;
}

template <typename T>
void make_hdr(const vamp_map_desc& r, double weight, double zinv, int d, unsigned char* out)
{
    ChanHdr<T> h;
    std::memset(&h, 0, sizeof h);
    h.wz = (T)(weight * std::pow(zinv, (double)(d - r.n_mapped)));
    for (int s = 0; s < r.n_mapped; ++s) {
        const int k = r.coord[s];
        h.mask |= 1u << k;
        h.slotpack |= (uint64_t)s << (4 * k);
        h.kinds |= (uint32_t)(r.kind[s] & 0xff) << (8 * s);
        T* sp = h.sp[s];
        if (r.kind[s] == VAMP_MAP_BW) {
            const double m = r.a[s], G = r.b[s], A = bw_A(m, G);
            sp[SP_M] = (T)m;
            sp[SP_G] = (T)G;
            sp[SP_A] = (T)A;
            sp[SP_G2] = (T)(G * G);
            sp[SP_INVG] = (T)(1.0 / G);
            sp[SP_GINVA] = (T)(G / A);
            sp[SP_INVA] = (T)(1.0 / A);
            sp[SP_T0] = (T)std::atan(m / G);
        } else if (r.kind[s] == VAMP_MAP_POW) {
            sp[SP_DEL] = (T)r.b[s];
            sp[SP_INVPOWN] = (T)pow_invN(r.b[s]);
        }
    }
    std::memcpy(out, &h, sizeof h);
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

bool build_setup(const vamp_config* cfg, Params& pr, Setup& S, std::string& why)
{
    if (!cfg) { why = "cfg is NULL"; return false; }
    const int d = cfg->d, K = cfg->n_channels, n = cfg->n_bins, P = cfg->n_peaks;
    if (d < 1 || d > DMAX) { why = "d must be in 1..16"; return false; }
    if (K < 1 || P < 1) { why = "need at least one channel and one peak"; return false; }
    if (n < 1 || n > MAX_BINS) { why = "n_bins must be in 1..256"; return false; }
    if (!cfg->channels || !cfg->peaks || !cfg->peak_weight) { why = "descriptor pointers are NULL"; return false; }
    if (!check_maps(cfg->channels, K, d, why) || !check_maps(cfg->peaks, P, d, why)) return false;
    if (!(cfg->gauss_sigma >= 0.0) || !std::isfinite(cfg->gauss_sigma)) { why = "gauss_sigma must be >= 0"; return false; }
    if (!(cfg->grid_alpha > 0.0) || !std::isfinite(cfg->beta)) { why = "grid_alpha must be > 0"; return false; }
    if (cfg->n_min < 1 || cfg->n_min > int64_t(0xffffffff)) { why = "n_min must be in 1..2^32-1"; return false; }
    if (cfg->gen_batch < 0 || cfg->gen_batch > (int64_t(1) << 24)) { why = "gen_batch out of range"; return false; }
    if (cfg->precision != VAMP_PREC_FP64 && cfg->precision != VAMP_PREC_FP32_EVAL) { why = "bad precision"; return false; }
    if (cfg->stratified != 0 && cfg->stratified != 1) { why = "stratified must be 0 or 1"; return false; }
    if (cfg->n_equiv < 0 || cfg->n_equiv > 65536 || (cfg->n_equiv > 0 && !cfg->equiv)) {
        why = "n_equiv must be in 0..65536 with a table"; return false;
    }
    if (cfg->n_equiv > 0 && (int64_t)K * d >= (int64_t(1) << 28)) { why = "too many grid rows for equivalences"; return false; }
    for (int e = 0; e < cfg->n_equiv; ++e) {
        const int32_t* r = cfg->equiv + (size_t)e * (2 + 2 * d);
        if (r[0] < 0 || r[0] >= K || r[1] < 0 || r[1] >= K) { why = "equivalence names a channel out of range"; return false; }
        unsigned seen = 0;
        for (int k = 0; k < d; ++k) {
            if (r[2 + k] < 0 || r[2 + k] >= d || (seen >> r[2 + k] & 1u)) {
                why = "equivalence axes must be a permutation of 0..d-1"; return false;
            }
            seen |= 1u << r[2 + k];
            if (r[2 + d + k] < VAMP_EQ_IDENTITY || r[2 + d + k] > VAMP_EQ_INVARIANT) {
                why = "equivalence kind must be 0..3"; return false;
            }
        }
    }
    for (int q = 0; q < P; ++q)
        if (!std::isfinite(cfg->peak_weight[q])) { why = "peak weights must be finite"; return false; }

    S.d = d; S.K = K; S.n = n; S.P = P;
    S.fp32 = cfg->precision == VAMP_PREC_FP32_EVAL;
    pr.d = d; pr.K = K; pr.n = n; pr.P = P;
    pr.key0 = (uint32_t)(cfg->seed & 0xffffffffu);
    pr.key1 = (uint32_t)(cfg->seed >> 32);
    pr.request = cfg->request_id;
    pr.n_min = cfg->n_min;
    pr.grid_alpha = cfg->grid_alpha;
    pr.beta = cfg->beta;
    pr.smooth = cfg->smooth;
    pr.omega_mode = cfg->omega_mode;
    pr.stratified = cfg->stratified;
    // equivalences regrouped by target grid row, list order kept (§3.5)
    S.eq_off.assign(cfg->n_equiv > 0 ? (size_t)K * d + 1 : 0, 0);
    S.eq_ent.clear();
    if (cfg->n_equiv > 0) {
        for (int row = 0; row < K * d; ++row) {
            const int c = row / d, k = row % d;
            S.eq_off[row] = (int32_t)S.eq_ent.size();
            for (int e = 0; e < cfg->n_equiv; ++e) {
                const int32_t* r = cfg->equiv + (size_t)e * (2 + 2 * d);
                if (r[0] == c) S.eq_ent.push_back(((r[1] * d + r[2 + k]) << 2) | r[2 + d + k]);
            }
        }
        S.eq_off[(size_t)K * d] = (int32_t)S.eq_ent.size();
    }
    pr.n_eq_ent = (int)S.eq_ent.size();
    // Gaussian factor exp(-(p-c)²/(2σ²)) / Z written as 2^-((p-c)² gk2) / Z,
    // gk2 = log2(e) / (2σ²); σ = 0 switches it off (factor 1)
    S.zinv = 1.0;
    pr.gcen = 0.0; pr.gk2 = 0.0; pr.gcen_f = 0.f; pr.gk2_f = 0.f;
    if (cfg->gauss_sigma > 0.0) {
        const double s = cfg->gauss_sigma, cc = cfg->gauss_centre;
        double Z;
        if (cfg->gauss_norm == VAMP_GAUSS_NORM_REAL_LINE) Z = s * std::sqrt(2.0 * M_PI);
        else Z = s * std::sqrt(M_PI / 2.0) * (std::erf((1.0 - cc) / (s * M_SQRT2)) + std::erf(cc / (s * M_SQRT2)));
        S.zinv = 1.0 / Z;
        pr.gcen = cc;
        pr.gk2 = M_LOG2E / (2.0 * s * s);
        pr.gcen_f = (float)cc;
        pr.gk2_f = (float)pr.gk2;
    }
    pr.matching = P == K;
    for (int q = 0; pr.matching && q < K; ++q)
        if (!same_maps(cfg->channels[q], cfg->peaks[q])) pr.matching = 0;
    pr.lay64 = make_layout_c<double>(d, n);
    pr.lay32 = make_layout_c<float>(d, n);

    S.hdr64.assign((size_t)K * pr.lay64.H, 0);
    S.hdr32.assign((size_t)K * pr.lay32.H, 0);
    for (int q = 0; q < K; ++q) {
        // with matching peaks the channel header carries the peak weight too
        const double w = pr.matching ? cfg->peak_weight[q] : 0.0;
        make_hdr<double>(cfg->channels[q], w, S.zinv, d, S.hdr64.data() + (size_t)q * pr.lay64.H);
        make_hdr<float>(cfg->channels[q], w, S.zinv, d, S.hdr32.data() + (size_t)q * pr.lay32.H);
    }
    S.pk64.assign((size_t)P * sizeof(MapRec<double>), 0);
    S.pk32.assign((size_t)P * sizeof(MapRec<float>), 0);
    for (int q = 0; q < P; ++q) {
        const MapRec<double> r64 = make_rec<double>(cfg->peaks[q], cfg->peak_weight[q], S.zinv, d);
        const MapRec<float> r32 = make_rec<float>(cfg->peaks[q], cfg->peak_weight[q], S.zinv, d);
        std::memcpy(S.pk64.data() + (size_t)q * sizeof r64, &r64, sizeof r64);
        std::memcpy(S.pk32.data() + (size_t)q * sizeof r32, &r32, sizeof r32);
    }
    return true;
}

Arena plan_arena(const Params& P)
{
    Arena A{};
    const size_t K = (size_t)P.K, rows = K * P.d;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += a256(bytes); return o; };
    A.edges64 = take(rows * (P.n + 1) * 8);
    A.lk64 = take(K * P.lay64.bytes);
    A.lk32 = take(K * P.lay32.bytes);
    A.alpha = take(K * 8);
    A.alpha32 = take(K * 4);
    A.shift = take(K * 8);
    A.acum = take(K * 8);
    A.nc = take(K * 8);
    A.pc = take((K + 1) * 8);
    A.D = take(rows * P.n * 8);
    A.csum = take(2 * K * 8);
    A.ic = take(K * 8);
    A.vc = take(K * 8);
    A.wc = take(K * 8);
    A.pk64 = take((size_t)P.P * sizeof(MapRec<double>));
    A.pk32 = take((size_t)P.P * sizeof(MapRec<float>));
    A.sc = take(sizeof(Scalars));
    A.nr = take(K * 8);
    A.spc = take(K * 8);
    A.coff = take((K + 1) * 8);
    A.qc = take(K * 8);
    A.eqoff = take(P.n_eq_ent > 0 ? (rows + 1) * 4 : 0);
    A.eqent = take((size_t)P.n_eq_ent * 4);
    A.bytes = off;
    return A;
}

void bind_arena(Params& P, unsigned char* b, const Arena& A)
{
    P.edges64 = (double*)(b + A.edges64);
    P.lk64 = b + A.lk64;
    P.lk32 = b + A.lk32;
    P.alpha = (double*)(b + A.alpha);
    P.alpha32 = (float*)(b + A.alpha32);
    P.shift = (double*)(b + A.shift);
    P.Acum = (double*)(b + A.acum);
    P.Nc = (int64_t*)(b + A.nc);
    P.Pc = (int64_t*)(b + A.pc);
    P.D = (double*)(b + A.D);
    P.csum = (double*)(b + A.csum);
    P.Ic = (double*)(b + A.ic);
    P.Vc = (double*)(b + A.vc);
    P.Wc = (double*)(b + A.wc);
    P.pk64 = (const MapRec<double>*)(b + A.pk64);
    P.pk32 = (const MapRec<float>*)(b + A.pk32);
    P.sc = (Scalars*)(b + A.sc);
    P.nr = (int64_t*)(b + A.nr);
    P.spc = (int64_t*)(b + A.spc);
    P.coff = (int64_t*)(b + A.coff);
    P.Qc = (double*)(b + A.qc);
    P.cellsum = nullptr;  // sized per pass by the context
    P.eq_off = P.n_eq_ent > 0 ? (const int32_t*)(b + A.eqoff) : nullptr;
    P.eq_ent = P.n_eq_ent > 0 ? (const int32_t*)(b + A.eqent) : nullptr;
}

cudaError_t upload_setup(const Params& P, const Setup& S, cudaStream_t s)
{
    cudaError_t e = cudaMemcpy2DAsync(P.lk64, P.lay64.bytes, S.hdr64.data(), P.lay64.H, P.lay64.H, P.K,
                                      cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(P.lk32, P.lay32.bytes, S.hdr32.data(), P.lay32.H, P.lay32.H, P.K,
                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void*)P.pk64, S.pk64.data(), S.pk64.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void*)P.pk32, S.pk32.data(), S.pk32.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && P.n_eq_ent > 0)
        e = cudaMemcpyAsync((void*)P.eq_off, S.eq_off.data(), S.eq_off.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && P.n_eq_ent > 0)
        e = cudaMemcpyAsync((void*)P.eq_ent, S.eq_ent.data(), S.eq_ent.size() * 4, cudaMemcpyHostToDevice, s);
    return e;
}

namespace {
void smem_for_budget(const Params& P, int fp32, size_t budget, int* tile, size_t* smem_int, size_t* smem_gen)
{
    const size_t S = (size_t)(fp32 ? P.lay32.bytes : P.lay64.bytes);
    const size_t ds = (size_t)P.d * P.n * 8;
    // FP64: each thread's power-law Jacobians of its call, one per coordinate,
    // where they fit beside one tile in a block's largest shared memory (the
    // kernel computes them per channel otherwise)
    size_t pw = fp32 ? 0 : (size_t)DMAX * PASS_THREADS * 8;
    int dev = 0, maxsm = 0;
    if (pw && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        SMEM_HEAD + 2 * S + ds + pw > (size_t)maxsm)
        pw = 0;
    const size_t fixed = SMEM_HEAD + ds + pw;
    long t = budget > fixed ? (long)((budget - fixed) / (2 * S)) : 1;
    if (t < 1) t = 1;
    if (t > P.K) t = P.K;
    *tile = (int)t;
    *smem_int = SMEM_HEAD + 2 * (size_t)t * S + ds + pw;
    *smem_gen = SMEM_HEAD + 2 * (size_t)t * S + pw;
}
}  // namespace

void pass_smem(const Params& P, int fp32, int* tile, size_t* smem_int, size_t* smem_gen)
{
    smem_for_budget(P, fp32, TILE_BUDGET, tile, smem_int, smem_gen);
}

void pass_smem_for(const Params& P, int fp32, int minb, int* tile, size_t* smem_int, size_t* smem_gen)
{
    // per-CTA share of the SM's shared memory, less the per-CTA reservation
    int dev = 0, per_sm = 0, reserved = 0;
    size_t budget = TILE_BUDGET;
    if (minb > 2 && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess)
        budget = std::min(budget, (size_t)(per_sm / minb - reserved));
    smem_for_budget(P, fp32, budget, tile, smem_int, smem_gen);
}

std::vector<const PassVariant*> pass_candidates(int fp32, int d, int n, int stratified, int K)
{
    static std::vector<PassVariant> all;
    static std::once_flag once;
    std::call_once(once, [] {
        add_pass_variants_f32_generic(all);
        add_pass_variants_f32_shapes(all);
        add_pass_variants_f64(all);
        add_pass_variants_union(all);
    });
    const bool uni = K > 0 && union_fits(fp32, d, K, n, stratified);
    std::vector<const PassVariant*> exact, generic, uexact, ugeneric;
    for (const PassVariant& v : all) {
        if (v.fp32 != fp32) continue;
        if (v.uni) {
            if (!uni) continue;
            if (v.D == d && v.NB == n) uexact.push_back(&v);
            else if (v.D == 0 && v.NB == 0) ugeneric.push_back(&v);
            continue;
        }
        if (v.D == d && v.NB == n && !stratified) exact.push_back(&v);
        else if (v.D == 0 && v.NB == 0) generic.push_back(&v);
    }
    for (const PassVariant* v : generic) exact.push_back(v);
    for (const PassVariant* v : uexact) exact.push_back(v);
    for (const PassVariant* v : ugeneric) exact.push_back(v);
    return exact;
}

cudaError_t ensure_smem(const void* fn, size_t bytes)
{
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess && fa.maxDynamicSharedSizeBytes < (int)bytes)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

}  // namespace vamp

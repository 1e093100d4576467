// vamp_union.cuh -- the FP32-eval pass kernel over per-coordinate interval
// tables ("union pass"), for problems with at most UNION_SLOTS channels.
//
// g(p) (Eq. 30) needs, for every channel c and coordinate k, the density of
// the bin of grid row (c, k) that holds x_{c,k} = φ_c^{-1}(p)_k.  The maps
// are increasing on [0, 1], so that bin is also the one whose image
// [φ_c(ξ_j), φ_c(ξ_{j+1})) holds p_k.  After every grid change the tables
// (vamp_union.cu) merge the images of all channels' edges on coordinate k
// into one sorted list U_k (rounded up to FP32, so that p >= U decides
// exactly as p >= φ_c(ξ_j) for an FP32 p); between two neighbouring values
// of U_k every channel's bin is fixed.  One interval search per coordinate
// then gives the K densities of a call as one 256-byte row, read coalesced.
// Only the Jacobians of the mapped coordinates remain per channel, and they
// need no inverse map: 1/φ' at p is Γ/(A((p-m)² + Γ²)) for a Breit-Wigner
// map and p^(-4/5)/5 for the power map x^5.
//
// Per batch of PASS_THREADS calls (one per thread), as k_pass where not said:
//   A  Philox words, channel, forward map, own term, integrand;
//   S  cell entries of p_k on every coordinate (their scans run between the
//      two halves of part J, so that the reads of U_k overlap it);
//   J  per channel c: α_c × the Jacobians of its mapped coordinates at p
//      (0 for the own and for switched-off channels) into shared memory, and
//      the matching integrand peak -- one quotient and two exponentials
//      per channel;
//   U  per warp, its 32 calls transposed, two calls per warp load: lane
//      (h, q) of half-warp h multiplies the densities of channels 4q..4q+3
//      of call 2j+h on every coordinate (one float4 of the call's row,
//      through L1, packed FP32x2 products) into the factors of J; a
//      reduce-scatter over each half-warp and one shuffle leave
//      Σ_c α_c g_c/φ'_c of call i in lane i;
//   C  weights; integration: shifted sums per warp and each call's w^2 added
//      to its d bins in global memory (FP64 reductions, no CTA barrier in
//      the batch loop); generation: acceptance and ordered compaction.
#pragma once

#include "vamp_pass.cuh"

namespace vamp {

constexpr int UNION_JSTR = UNION_SLOTS + 2;  // floats per call row of the channel factors (8-byte rows, 2-way banks)

// A channel's terms for part J, copied into shared memory once per CTA:
// α_c 0.2^npw; the matching peak's weight times the product of its
// power-law normalisations 1/powN; the product of its Breit-Wigner
// numerators Γ/A; and its mapped coordinates, the nbw Breit-Wigner ones
// first (m, Γ², -, k), then the npw power-law ones (δ, -, -, k), so that
// part J runs two loops of uniform trip count with no test of the map kind.
// A channel's factors are formed with one quotient and two exponentials:
// its Breit-Wigner Jacobians Γ/(A((p-m)² + Γ²)) as the constant over the
// product of the denominators (each at least Γ² >= 1e-8, so the product of
// four stays a normal FP32 number), its power-law Jacobians
// Π 0.2 p^(-4/5) = 0.2^npw 2^(-0.8 Σ log2 p), and the peak's power-law
// factors Π (p + δ)^(-4/5) joined to its Gaussian exponent.
struct UnionChan {
    float alpha, wz, jc;  // α_c 0.2^npw, the peak weight Π 1/powN, Π_BW Γ/A
    int nslot;            // nbw | (nbw + npw) << 8: the Breit-Wigner slots and the end of the power-law ones
    float4 slot[MAXMAP];  // {c0, c1, -, bits of k}
};
static_assert(sizeof(UnionChan) == 80, "UnionChan layout");

// Shared-memory layout of the union kernel (bytes from the start).
struct UnionSmem {
    int ds, js, ps, us, ch, bytes;
};
__host__ __device__ constexpr int union_pstride(int DM) { return DM | 1; }
__host__ __device__ constexpr UnionSmem union_smem_layout(int DM, int d, int n, int mode)
{
    const int nw = PASS_THREADS / 32;
    const int ds = SMEM_HEAD;  // no shared d-values: calls add theirs to global memory
    const int js = ds;
    const int ps = js + nw * 32 * UNION_JSTR * 4;
    const int us = ps + round_up(PASS_THREADS * union_pstride(DM) * 4, 16);
    const int ch = us + round_up(nw * DM * 32 * 2, 16);
    const int bytes = ch + UNION_SLOTS * (int)sizeof(UnionChan);
    return UnionSmem{ds, js, ps, us, ch, bytes};
}

// One float4 of a density row, through L1 with the evict_unchanged
// priority.  Measured on the collider pass with float2 loads (1e7 calls,
// after an L2 flush / warm): 5.61 / 5.59 ms, against 5.91 / 5.62 ms
// without allocating in L1, 5.93 / 5.62 ms with evict_first and
// 5.75 / 5.73 ms with the default policy: calls cluster, so the warps of
// an SM share rows.
__device__ __forceinline__ float4 ld_row(const float4* p)
{
    float4 v;
    asm("ld.global.nc.L1::evict_unchanged.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

// Cell entry of x on coordinate k (the first step of union_interval).
__device__ __forceinline__ uint32_t union_cell_entry(const Params& P, int k, float x)
{
    const int q = min(Prec<float>::cell(x, UNION_LCELLS), UNION_CELLS - 1);
    return __ldg(P.uC + (size_t)k * UNION_CELLS + q);
}

// Interval of x in U_k from x's cell entry e: the index of the largest
// U_k[u] <= x (0 if none).
__device__ __forceinline__ int union_interval(const Params& P, int k, float x, uint32_t e)
{
    const int base = (int)(e & 0xffffu), span = (int)(e >> 16);
    const float* Uk = P.uU + (size_t)k * P.uMax + base;
    // most cells hold at most one value of U_k: one comparison, no loop
    int t = (span > 0 && __ldg(Uk) <= x) ? 1 : 0;
    if (t == 1 && span > 1)
        while (t < span && __ldg(Uk + t) <= x) ++t;
    return max(base + t - 1, 0);
}

template <int MODE, int D_, int NB_, int MINB>
__global__ void __launch_bounds__(PASS_THREADS, MINB) k_union(Params P, PassArgs A)
{
    using SH = Shape<float, D_, NB_>;
    constexpr int DM = SH::DM;
    constexpr int PSTR = union_pstride(DM);
    constexpr int NW = PASS_THREADS / 32;
    static_assert(union_smem_layout(DM, 1, 1, MODE).us % 16 == 0, "part U reads the intervals as 16-byte words");
    extern __shared__ __align__(128) unsigned char smem[];
    SmemHead& H = *reinterpret_cast<SmemHead*>(smem);
    const SH sh(P.lay32, P.d, P.n);
    const int d = sh.d(), n = sh.n(), dn = d * n, K = P.K;
    const UnionSmem L = union_smem_layout(DM, d, n, MODE);
    float* Js = reinterpret_cast<float*>(smem + L.js);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float* Jw = Js + wid * 32 * UNION_JSTR;                                       // factors of this warp's calls
    float* Pt = reinterpret_cast<float*>(smem + L.ps) + tid * PSTR;                // p of this thread's call
    uint16_t* Uw = reinterpret_cast<uint16_t*>(smem + L.us) + wid * DM * 32;     // intervals of the warp's calls
    constexpr int B = PASS_THREADS;

    UnionChan* ucs = reinterpret_cast<UnionChan*>(smem + L.ch);
    // channel slots >= K keep factor 0 (their density rows are 0 as well)
    for (int i = tid; i < NW * 32 * UNION_JSTR; i += PASS_THREADS) Js[i] = 0.f;
    // part J's channel terms from the lookup-block headers (one thread per
    // channel; mapped coordinates of other kinds carry no factor)
    for (int c = tid; c < K; c += PASS_THREADS) {
        const ChanHdr<float>* h = reinterpret_cast<const ChanHdr<float>*>(P.lk32 + (size_t)c * sh.bytes());
        const uint32_t mask = h->mask, kinds = h->kinds;
        const uint64_t slotpack = h->slotpack;
        int nb = 0, np = 0;
        float wz = h->wz, jc = 1.f, a5 = 1.f;
        for (int pass = 0; pass < 2; ++pass) {
            for (uint32_t m = mask; m; m &= m - 1u) {
                const int k = __ffs(m) - 1;
                const int s = (int)((slotpack >> (4 * k)) & 0xFu);
                const int kind = (kinds >> (8 * s)) & 0xff;
                const float* sp = h->sp[s];
                if (pass == 0 && kind == MAP_BW) {
                    ucs[c].slot[nb++] = make_float4(sp[SP_M], sp[SP_G2], 0.f, __int_as_float(k));
                    jc *= sp[SP_GINVA];
                } else if (pass == 1 && kind == MAP_POW) {
                    ucs[c].slot[nb + np++] = make_float4(sp[SP_DEL], 0.f, 0.f, __int_as_float(k));
                    wz *= sp[SP_INVPOWN];
                    a5 *= 0.2f;
                }
            }
        }
        ucs[c].alpha = P.alpha32[c] * a5;
        ucs[c].wz = wz;
        ucs[c].jc = jc;
        ucs[c].nslot = nb | ((nb + np) << 8);
    }
    __syncthreads();

    // ---- work of this CTA (as k_pass, one call per thread) -------------------
    int64_t r0 = 0, r1 = 0, nbatch = 0;
    if (MODE == 0) {
        const int64_t N = P.sc->n_total;
        r0 = N * blockIdx.x / gridDim.x;
        r1 = N * (blockIdx.x + 1) / gridDim.x;
        for (int64_t i = r0; i < r1;) {
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

    double wm = 0.0, s1 = 0.0, s2 = 0.0;
    bool bad = false;
    int64_t i0 = r0;
    int cseg = -1;
    int64_t seg_end = 0;
    double sft = 0.0;
    int64_t chunk = blockIdx.x;
    const float gc = P.gcen_f, k2 = P.gk2_f;
    const bool with_f = P.matching != 0;

    for (int64_t bt = 0; bt < nbatch; ++bt) {
        int64_t base, end;
        if (MODE == 0) {
            if (i0 >= seg_end || cseg < 0) {
                cseg = find_channel(P.Pc, K, i0);
                seg_end = min(r1, P.Pc[cseg + 1]);
                sft = P.shift[cseg];
            }
            base = i0;
            end = min(seg_end, i0 + B);
        } else {
            base = chunk * B;
            end = min(A.batch, base + B);
        }

        // ---- A: own channel's forward map, own term, integrand ------------------
        Calls<float, 1, DM> C;
        phase_a<float, MODE, 1>(P, sh, A.field, base, end, cseg, C);

        // ---- S: p to shared memory and its interval on every coordinate --------
#pragma unroll
        for (int k = 0; k < DM; ++k)
            if (sh.has(k)) Pt[k] = C.p[0][k];
        // cell entries now, the scan after part J (their latency hides behind it)
        uint32_t ce[DM];
#pragma unroll
        for (int k = 0; k < DM; ++k) ce[k] = sh.has(k) ? union_cell_entry(P, k, C.p[0][k]) : 0u;

        // ---- J: α_c times the Jacobians of channel c's mapped coordinates ------
        const int own = MODE == 0 ? cseg : C.cq[0];
        const float Aq = C.Aexp[0];
        float f = C.f[0];
        // two halves of the channels; the interval scans (whose cell entries
        // were loaded above) run between them, so that their reads of U_k
        // overlap the second half
        for (int half = 0; half < 2; ++half) {
            const int c_lo = half == 0 ? 0 : K / 2, c_hi = half == 0 ? K / 2 : K;
#pragma unroll 4
            for (int c2 = c_lo; c2 < c_hi; ++c2) {
                const UnionChan& ch = ucs[c2];
                const int nb = ch.nslot & 0xff, ne = ch.nslot >> 8;
                float den = 1.f, as = 0.f, lp = 0.f, lq = 0.f;
#pragma unroll 1
                for (int s = 0; s < nb; ++s) {
                    const float4 r = ch.slot[s];
                    const float pk = Pt[__float_as_int(r.w)];
                    const float dp = pk - r.x;
                    den *= fmaf(dp, dp, r.y);
                    const float u = pk - gc;
                    as = fmaf(u, u, as);  // Σ (p_k - c)², times k2 once per channel
                }
#pragma unroll 1
                for (int s = nb; s < ne; ++s) {
                    const float4 r = ch.slot[s];
                    const float pk = Pt[__float_as_int(r.w)];
                    lp += Prec<float>::lg2(pk);
                    if (with_f) lq += Prec<float>::lg2(pk + r.x);
                    const float u = pk - gc;
                    as = fmaf(u, u, as);  // Σ (p_k - c)², times k2 once per channel
                }
                const float jb = Prec<float>::div(ch.jc, den);  // Π_BW 1/φ' = Π_BW Γ/A over Π_BW ((p-m)² + Γ²)
                const float J = jb * Prec<float>::exp2_(-0.8f * lp);  // lp = 0 without power-law slots
                const float a = ch.alpha;
                Jw[lane * UNION_JSTR + c2] = a != 0.f ? a * J : 0.f;  // the own channel's is cleared below
                if (with_f) f += ch.wz * Prec<float>::exp2_(fmaf(-0.8f, lq, fmaf(as, k2, -Aq))) * jb;
            }
            if (half == 0) {
                // ---- S (end): intervals from the cell entries --------------------
#pragma unroll
                for (int k = 0; k < DM; ++k)
                    if (sh.has(k)) Uw[k * 32 + lane] = (uint16_t)union_interval(P, k, Pt[k], ce[k]);
            }
        }
        // the own channel's term is in g already (phase A)
        if ((unsigned)own < (unsigned)K) Jw[lane * UNION_JSTR + own] = 0.f;
        __syncwarp();

        // ---- U: densities of the warp's calls: half-warp h takes calls 2j+h
        // (j = 0..15), its lane q channels 4q..4q+3 --------------------------
        {
            const int h = lane >> 4, q = lane & 15;
            float2 lo[16], hi[16];  // channels 4q, 4q+1 and 4q+2, 4q+3 of call 2j+h
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float* jr = Jw + (2 * j + h) * UNION_JSTR + 4 * q;
                lo[j] = *reinterpret_cast<const float2*>(jr);
                hi[j] = *reinterpret_cast<const float2*>(jr + 2);
            }
            // the intervals of calls 2j and 2j+1 share 32-bit word j (low and
            // high half); a lane takes its half with one byte permute
            const uint32_t sel = h ? 0x4432u : 0x4410u;
#pragma unroll 1
            for (int k = 0; k < d; ++k) {
                const float4* row = reinterpret_cast<const float4*>(P.uD + (size_t)k * P.uMax * UNION_SLOTS) + q;
                // the warp's 32 intervals of coordinate k: 64 bytes at a 16-byte
                // boundary (the layout rounds every region to 16 bytes and a
                // warp's block is DM * 64 bytes), four broadcast loads
                const uint4* uw = reinterpret_cast<const uint4*>(Uw + k * 32);
#pragma unroll
                for (int j4 = 0; j4 < 4; ++j4) {
                    const uint4 w = uw[j4];
                    const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = 4 * j4 + t;
                        const uint32_t u = __byte_perm(wv[t], 0u, sel);  // interval of call 2j+h
                        const float4 r = ld_row(row + (size_t)u * (UNION_SLOTS / 4));
                        lo[j] = __fmul2_rn(lo[j], make_float2(r.x, r.y));  // packed FP32x2
                        hi[j] = __fmul2_rn(hi[j], make_float2(r.z, r.w));
                    }
                }
            }
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = (lo[j].x + lo[j].y) + (hi[j].x + hi[j].y);
            // reduce-scatter within the half-warp: in the step of width s
            // each lane trades half of its partial sums with lane ^ s (the
            // lane with bit s set keeps the upper half), so that after four
            // steps v[0] of lane (h, q) is the sum over the half for call 2q+h
#pragma unroll
            for (int s = 8; s >= 1; s >>= 1) {
                const bool up = (q & s) != 0;
#pragma unroll
                for (int j = 0; j < s; ++j) {
                    const float send = up ? v[j] : v[j + s];
                    const float keep = up ? v[j + s] : v[j];
                    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
                }
            }
            // call `lane` = 2q+h sits in lane 16h + q
            C.g[0] += __shfl_sync(0xffffffffu, v[0], ((lane & 1) << 4) | (lane >> 1));
        }
        C.f[0] = f;
#pragma unroll
        for (int k = 0; k < DM; ++k)
            if (sh.has(k)) C.p[0][k] = Pt[k];
        __syncwarp();  // the next batch overwrites this warp's factors and intervals

        // ---- C: weights and accumulation ----------------------------------------
        if (MODE == 0) {
            // weight, shifted sums and d-values (Eq. 15): each call adds its
            // w^2 to its d bins in global memory (FP64 reductions, no wait);
            // the warp's shifted sums go out once per batch
            if (C.valid[0]) {
                double w = C.g[0] > 0.f ? (double)(C.f[0] / C.g[0]) : 0.0;
                if (!isfinite(w)) { bad = true; w = 0.0; }
                const double dv = w - sft;
                s1 = dv;
                s2 = dv * dv;
                wm = fmax(wm, fabs(w));  // signed integrands: w_max bounds |w|
                const double w2 = w * w;
                double* Dc = P.D + (size_t)cseg * dn;
#pragma unroll
                for (int k = 0; k < DM; ++k)
                    if (sh.has(k)) atomicAdd(&Dc[k * n + ((C.jp[0][k >> 2] >> (8 * (k & 3))) & 0xff)], w2);
            } else {
                s1 = s2 = 0.0;
            }
            s1 = warp_sum(s1);
            s2 = warp_sum(s2);
            if (lane == 0) {
                atomicAdd(&P.csum[2 * cseg], s1);
                atomicAdd(&P.csum[2 * cseg + 1], s2);
            }
            i0 = end;
        } else {
            phase_c_gen<float, 1>(P, A, sh, C, chunk, base, H.wcnt, H.woff, &H.round_total, wm, bad);
            chunk += gridDim.x;
        }
    }

    if (bad) atomicOr(&P.sc->err, ERR_NONFINITE);
    block_max_to(H, wm, MODE == 0 ? &P.sc->wmax_bits : &P.sc->gen_bmax_bits);
}

template <int D_, int NB_, int MINB>
cudaError_t union_launch_t(const Params& P, int mode, const PassArgs& A, int grid, size_t smem, cudaStream_t s)
{
    if (mode) k_union<1, D_, NB_, MINB><<<grid, PASS_THREADS, smem, s>>>(P, A);
    else k_union<0, D_, NB_, MINB><<<grid, PASS_THREADS, smem, s>>>(P, A);
    return cudaGetLastError();
}

template <int D_, int NB_, int MINB = 2>
PassVariant make_union_variant()
{
    PassVariant v;
    v.fp32 = 1;
    v.cpt = 1;
    v.D = D_;
    v.NB = NB_;
    v.minb = MINB;
    v.family = "k_union";
    v.uni = 1;
    v.fn[0] = (const void*)k_union<0, D_, NB_, MINB>;
    v.fn[1] = (const void*)k_union<1, D_, NB_, MINB>;
    v.launch = &union_launch_t<D_, NB_, MINB>;
    return v;
}

}  // namespace vamp

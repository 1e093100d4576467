// vamp_union.cu -- interval tables of the union pass (vamp_union.cuh) and
// its kernel variants.
//
// After every change of the grids (creation, rebinning, state upload) the
// tables are rebuilt from the FP64 master grids, coordinate by coordinate:
//   k_union_images  image of every edge under its channel's map,
//                   v = φ_c(ξ_{c,k,j}) in FP64 (the forward map's formula),
//                   rounded up to FP32: for an FP32 p, p >= v32 exactly when
//                   p >= v, so comparing p with the images decides the bin
//                   as comparing φ_c^{-1}(p) with the edges does;
//   k_union_sort    the K (n+1) images of a coordinate sorted (bitonic
//                   network in shared memory) and made distinct: U_k;
//   k_union_cells   for each of UNION_CELLS equal cells [q/L, (q+1)/L) the
//                   count of U_k values <= q/L and the count inside the cell;
//   k_union_rows    for each interval [U_k[u], U_k[u+1]) and channel c the
//                   FP32 density 1/(nΔx) of the bin of row (c, k) whose image
//                   holds it: the largest j <= n-1 with image_j <= U_k[u]
//                   (bin 0 below the first image), from the lookup block.
#include "vamp_union.cuh"

#include <algorithm>

namespace vamp {

namespace {

__global__ void k_union_images(Params P)
{
    const int d = P.d, K = P.K, n1 = P.n + 1;
    const int64_t tot = (int64_t)d * K * n1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % n1);
        const int c = (int)((t / n1) % K);
        const int k = (int)(t / ((int64_t)n1 * K));
        const double e = P.edges64[((size_t)c * d + k) * n1 + j];
        const ChanHdr<double>* h = reinterpret_cast<const ChanHdr<double>*>(P.lk64 + (size_t)c * P.lay64.bytes);
        double v = e;
        if ((h->mask >> k) & 1u) {
            const int s = (int)((h->slotpack >> (4 * k)) & 0xFu);
            const int kind = (h->kinds >> (8 * s)) & 0xff;
            const double* sp = h->sp[s];
            if (kind == MAP_BW) {
                v = sp[SP_M] + sp[SP_G] * Prec<double>::tan_(sp[SP_A] * e - sp[SP_T0]);
            } else if (kind == MAP_POW) {
                const double e2 = e * e, e4 = e2 * e2;
                v = e4 * e;
                if (v < Prec<double>::tiny()) v = Prec<double>::tiny();
            }
        }
        P.uImg[t] = __double2float_ru(v);  // [k][c][j]
    }
}

constexpr int SORT_THREADS = 1024;

// One block per coordinate; dynamic shared memory: the padded image list.
__global__ void __launch_bounds__(SORT_THREADS) k_union_sort(Params P, int np)
{
    extern __shared__ float sv[];
    __shared__ int wsum[SORT_THREADS / 32];
    const int k = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int m = P.K * (P.n + 1);
    const float* src = P.uImg + (size_t)k * m;
    for (int i = tid; i < np; i += SORT_THREADS) sv[i] = i < m ? src[i] : INFINITY;
    __syncthreads();
    // bitonic network, ascending
    for (int size = 2; size <= np; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < np / 2; i += SORT_THREADS) {
                const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const float a = sv[lo], b = sv[hi];
                if ((a > b) == up) { sv[lo] = b; sv[hi] = a; }
            }
            __syncthreads();
        }
    }
    // distinct values, in order: each thread a contiguous run, block scan of
    // the run counts
    const int per = (m + SORT_THREADS - 1) / SORT_THREADS;
    const int i0 = min(tid * per, m), i1 = min(i0 + per, m);
    int cnt = 0;
    for (int i = i0; i < i1; ++i) cnt += (i == 0 || sv[i] != sv[i - 1]) ? 1 : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = wsum[lane];
        int iw = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, iw, o);
            if (lane >= o) iw += y;
        }
        wsum[lane] = iw - w;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    int pos = wsum[wid] + incl - cnt;
    float* U = P.uU + (size_t)k * P.uMax;
    for (int i = i0; i < i1; ++i)
        if (i == 0 || sv[i] != sv[i - 1]) U[pos++] = sv[i];
    if (tid == SORT_THREADS - 1) P.uNU[k] = wsum[wid] + incl;
}

// count of U[0..nu) <= x (le) or < x (!le)
__device__ __forceinline__ int count_below(const float* U, int nu, float x, bool le)
{
    int lo = 0, hi = nu;  // first index whose value is > x (le) or >= x (!le)
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const bool below = le ? (U[mid] <= x) : (U[mid] < x);
        if (below) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_union_cells(Params P)
{
    const int k = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= UNION_CELLS) return;
    const float* U = P.uU + (size_t)k * P.uMax;
    const int nu = P.uNU[k];
    const float step = 1.0f / (float)UNION_CELLS;  // a power of two: q step is exact
    const int base = count_below(U, nu, (float)q * step, true);
    const int span = q == UNION_CELLS - 1 ? nu - base : count_below(U, nu, (float)(q + 1) * step, false) - base;
    P.uC[(size_t)k * UNION_CELLS + q] = (uint32_t)base | ((uint32_t)span << 16);
}

constexpr int ROWS_PER_BLOCK = 64;

// Block (u-range, coordinate); dynamic shared memory: the K (n+1) images of
// the coordinate.
__global__ void k_union_rows(Params P)
{
    extern __shared__ float im[];
    const int k = blockIdx.y;
    const int nu = P.uNU[k];
    const int u0 = blockIdx.x * ROWS_PER_BLOCK;
    if (u0 >= nu) return;
    const int K = P.K, n = P.n, n1 = n + 1;
    const float* src = P.uImg + (size_t)k * K * n1;
    for (int i = threadIdx.x; i < K * n1; i += blockDim.x) im[i] = src[i];
    __syncthreads();
    const float* U = P.uU + (size_t)k * P.uMax;
    const BlkLayout& L = P.lay32;
    for (int t = threadIdx.x; t < ROWS_PER_BLOCK * UNION_SLOTS; t += blockDim.x) {
        const int u = u0 + t / UNION_SLOTS, c = t % UNION_SLOTS;
        if (u >= nu) break;
        float val = 0.f;
        if (c < K) {
            const float x = U[u];
            const float* e = im + c * n1;
            int lo = 0, hi = n - 1;  // largest j in [0, n-1] with e[j] <= x (0 if none)
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (e[mid] <= x) lo = mid; else hi = mid - 1;
            }
            const float* dn = reinterpret_cast<const float*>(P.lk32 + (size_t)c * L.bytes + L.H + (size_t)k * L.R +
                                                             (size_t)L.Es * sizeof(float));
            val = dn[lo];
        }
        P.uD[((size_t)k * P.uMax + u) * UNION_SLOTS + c] = val;
    }
}

int sort_width(int m)
{
    int np = 2;
    while (np < m) np <<= 1;
    return np;
}

}  // namespace

bool union_fits(int fp32, int d, int K, int n, int stratified)
{
    return fp32 && !stratified && d >= 1 && K >= 1 && K <= UNION_SLOTS && K * (n + 1) <= UNION_MAXV;
}

size_t union_bytes(int d, int K, int n)
{
    const size_t m = (size_t)K * (n + 1);
    auto a256 = [](size_t v) { return (v + 255) & ~size_t(255); };
    return a256(d * m * 4) + a256(d * m * 4) + a256((size_t)d * 4) + a256((size_t)d * UNION_CELLS * 4) +
           a256(d * m * UNION_SLOTS * 4);
}

void bind_union(Params& P, unsigned char* base)
{
    const size_t m = (size_t)P.K * (P.n + 1);
    const int d = P.d;
    auto a256 = [](size_t v) { return (v + 255) & ~size_t(255); };
    P.uMax = (int)m;
    if (!base) {
        P.uImg = P.uU = P.uD = nullptr;
        P.uNU = nullptr;
        P.uC = nullptr;
        return;
    }
    unsigned char* q = base;
    P.uImg = reinterpret_cast<float*>(q); q += a256(d * m * 4);
    P.uU = reinterpret_cast<float*>(q); q += a256(d * m * 4);
    P.uNU = reinterpret_cast<int*>(q); q += a256((size_t)d * 4);
    P.uC = reinterpret_cast<uint32_t*>(q); q += a256((size_t)d * UNION_CELLS * 4);
    P.uD = reinterpret_cast<float*>(q);
}

cudaError_t launch_union_build(const Params& P, cudaStream_t s)
{
    const int d = P.d, m = P.K * (P.n + 1);
    const int np = sort_width(m);
    const size_t sort_smem = (size_t)np * 4, rows_smem = (size_t)m * 4;
    cudaError_t e = ensure_smem((const void*)k_union_sort, sort_smem);
    if (e == cudaSuccess) e = ensure_smem((const void*)k_union_rows, rows_smem);
    if (e != cudaSuccess) return e;
    const int64_t tot = (int64_t)d * m;
    k_union_images<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(P);
    k_union_sort<<<d, SORT_THREADS, sort_smem, s>>>(P, np);
    k_union_cells<<<dim3(UNION_CELLS / 256, d), 256, 0, s>>>(P);
    k_union_rows<<<dim3((m + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK, d), 256, rows_smem, s>>>(P);
    return cudaGetLastError();
}

size_t union_pass_smem(const Params& P, const PassVariant& v, int mode)
{
    const int DM = v.D > 0 ? v.D : DMAX;
    return (size_t)union_smem_layout(DM, P.d, P.n, mode).bytes;
}

void add_pass_variants_union(std::vector<PassVariant>& v)
{
    v.push_back(make_union_variant<14, 100, 2>());
    v.push_back(make_union_variant<0, 0, 2>());
}

}  // namespace vamp

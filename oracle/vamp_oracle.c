/*
 * vamp_oracle.c -- plain, slow, FP64 CPU oracle of the doubly adaptive
 * multi-channel integrator (VAMP) of arXiv:1811.09711, §3.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load, link or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two meet only in the seeded problem
 * arrays handed to both.
 *
 * Every step is written in the order and notation of the paper:
 *   - §3.2  VEGAS step map G, density g(x) = prod_k 1/(n Δx_{k j_k}) (Eq. 12),
 *           rebinning measure m_j (Eq. 14) from bin weights ω_j (Eq. 15);
 *   - §3.1  estimators E_N, V_N (Eqs. 5, 6, 10, 11);
 *   - §3.4  channel weights α_c (Eq. 16), update α_c ω_c^β / Σ α ω^β (Eq. 25),
 *           integer N_c with a lower threshold;
 *   - §3.5  per-channel grids g_c (Eq. 26), multi-channel density
 *           g(p) = Σ_c α_c g_c(x_c)/φ'_c(x_c) with x_c = φ_c^{-1}(p) (Eq. 30),
 *           weight w = f(p)/g(p) (Eq. 29, ρ = 1) and estimator (Eq. 31);
 *           the per-call work order (map the selected channel, evaluate f,
 *           invert all other channels, accumulate);
 *           event generation from the final grids with a random channel
 *           chosen by α and rejection against the maximum weight (§2, Eq. 2);
 *   - §4.4  reproducible, communication-free random streams: here the
 *           counter-based Philox4x32-10 of Salmon et al. (SC'11).
 *
 * Readings where the paper is silent (each one also stated where it is used):
 *   R1  ρ = 1; D_{c,k,j} = Σ w² over calls of channel c with x_{c,k} in bin j.
 *   R2  m_j limits: r_j = 0 -> 0; |r_j - 1| < 1e-12 -> 1; Σω = 0 -> axis kept.
 *   R3  optional 3-point smoothing of D (off by default).
 *   R4  rebinning = continuous inversion of the cumulative of m over the old
 *       piecewise-linear grid; first edge 0, last edge 1.
 *   R5  α update: ω_c = V_c (or the second moment); channels without variance
 *       keep α_c; channels whose calls all gave w = 0 are switched off.
 *   R6  N_c = max(N_min, floor(α_c N)) for α_c > 0, else 0.
 *   R7  x_c = φ_c^{-1}(p) in Eq. 30 (the printed subscript is garbled).
 *   R8  error of I is sqrt(σ²) with σ² = Σ α_c² V_c / N_c.
 *   R9  combination of iterations: inverse-variance weighted mean, χ²/dof.
 *   R10 u = (X + 1/2) 2^-32; forward bin j and fraction from (2X+1) n.
 *   R11 bin search: largest j with ξ_j <= x, clamped to [0, n-1].
 *   R12 generation: w_max from the last integration pass, raised between
 *       batches; accept iff u w_max < |w| (R19); overweights counted.
 *   R13 per-channel sums shifted by the previous pass's channel mean.
 *   R14 synthetic integrand factors normalised on [0,1] (or the real line).
 *   R15 power map p = x^5 with p clamped to >= the smallest normal double.
 *   R16 pseudo-stratified sampling (§3.3, optional): per channel, n_r cells
 *       per r axis, the largest m (<= 2^20) with 2 m^d <= N_c; C = n_r^d
 *       cells; s = floor(N_c / C) points per cell; the channel samples
 *       N_c = s C calls.  Local call l lies in cell floor(l / s), whose
 *       base-n_r digits a_k place r_k = (a_k + u_k) / n_r; the forward bin
 *       and fraction come from the integer (2^33 a_k + 2X + 1) n over
 *       n_r 2^33 (R10 is the case n_r = 1).  Generation stays importance
 *       sampling.
 *   R17 stratified variance: the per-call variance entering σ² (R8) and the
 *       α update is the mean over the channel's cells of the cells' sample
 *       variances, [Σ d² - Σ_cells (Σ_cell d)² / s] / (C (s - 1)) with
 *       d = w - s_c (R13); 0 for s < 2.
 *   R18 channel equivalences (§3.5, optional): the bin weights that the
 *       rebinning of channel c uses are its d-values D_c (R1) plus, for each
 *       listed equivalence (c <- c', π, mode per axis), the d-values of axis
 *       π(k) of c': identity adds D_{c',π(k),j}; invert adds D_{c',π(k),n-1-j}
 *       (the paper's "d - j" read as the mirrored bin of an n-bin axis);
 *       symmetric adds the mean of the two; invariant sets the row to 1 (the
 *       rebinning then keeps the axis).  All sums read the pass's own D (the
 *       equivalences act at once, not one after another), terms add in list
 *       order, and c' = c is allowed.
 *   R19 signed integrands (§3.1 allows f < 0, e.g. at NLO): the estimators
 *       and d-values are unchanged (D sums w² anyway); w_max is the largest
 *       |w|; generation accepts with probability |w| / w_max and the event
 *       keeps w with its sign; overweights are |w| > w_max.  The pass's
 *       efficiency stays Eq. 2, ⟨w⟩ / w_max: the net yield after the signs
 *       cancel.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_MAPPED 4
#define OR_MAX_HIST 4096
#define OR_MAX_D 64

enum { OR_MAP_ID = 0, OR_MAP_BW = 1, OR_MAP_POW = 2 };
enum { OR_EQ_IDENTITY = 0, OR_EQ_INVERT = 1, OR_EQ_SYMMETRIC = 2, OR_EQ_INVARIANT = 3 };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_STATE = 2, OR_ERR_NUMERIC = 3, OR_ERR_MEM = 4 };

/* Problem as handed over by the harness (arrays are copied). */
typedef struct {
    int32_t d, n_channels, n_bins;
    const int32_t *ch_nmap, *ch_coord, *ch_kind; /* K, K*4, K*4 */
    const double *ch_a, *ch_b;                   /* K*4 */
    int32_t n_peaks;
    const double *pk_w;                          /* P */
    const int32_t *pk_nmap, *pk_coord, *pk_kind; /* P, P*4, P*4 */
    const double *pk_a, *pk_b;                   /* P*4 */
    double gauss_sigma, gauss_centre;
    int32_t gauss_norm;                          /* 0: real line, 1: [0,1] */
    uint64_t seed;
    uint32_t request_id;
    double grid_alpha, beta;
    int64_t n_min;
    int32_t smooth, omega_mode;
    int64_t gen_batch;
    int32_t stratified;                          /* R16 */
    int32_t n_equiv;                             /* R18 */
    const int32_t *equiv;                        /* n_equiv records: c, c', π[d], mode[d] */
} or_problem;

/* Neumaier-compensated sum. */
typedef struct { double s, c; } ksum;
static void ks_add(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}
static double ks_val(const ksum *k) { return k->s + k->c; }

typedef struct {
    int32_t nmap;
    int32_t coord[OR_MAX_MAPPED], kind[OR_MAX_MAPPED];
    double a[OR_MAX_MAPPED], b[OR_MAX_MAPPED];
    /* derived constants of the maps / factors (§3.4 mappings) */
    double bwA[OR_MAX_MAPPED], bwT0[OR_MAX_MAPPED], powN[OR_MAX_MAPPED];
    int32_t slot_of[OR_MAX_D]; /* coordinate -> slot, or -1 */
} or_maps;

typedef struct or_ctx {
    int d, K, n, P;
    or_maps *ch, *pk;
    double *pk_w;
    double gsig, gcen, gZ;
    int gnorm;
    uint32_t key[2];
    uint32_t request;
    double grid_alpha, beta;
    int64_t n_min;
    int smooth, omega_mode;
    int64_t gen_batch;
    /* state */
    double *edges;   /* K*d*(n+1): ξ_{c,k,j} */
    double *alpha;   /* K */
    double *shift;   /* K: s_c (R13) */
    int64_t *Nc, *Pc; /* K, K+1 */
    int stratified;   /* R16 */
    int64_t *nr, *spc, *Cc; /* K each: cells per axis, points per cell, cells */
    int64_t n_total;
    double *D;       /* K*d*n */
    int n_eq;        /* R18 */
    int32_t *eq;     /* n_eq * (2 + 2d) */
    double *Dp;      /* K*d*n: bin weights after the equivalences */
    double *Ic, *Vc, *Wc; /* K */
    int have_pass;
    double wmax;
    int n_hist;
    double hist_I[OR_MAX_HIST], hist_V[OR_MAX_HIST];
    int hist_comb[OR_MAX_HIST];
    double comb_I, comb_sigma, comb_chi2;
} or_ctx;

/* ------------------------------------------------------------------ */
/* §4.4: counter-based random numbers, Philox4x32-10 (Salmon et al.).  */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random words of one call: word w lives in block w/4, lane w%4 of the
 * Philox output for counter (call, block, stream field, request). */
static void call_words(const or_ctx *o, uint32_t call, uint32_t field, int nwords, uint32_t *X)
{
    for (int b = 0; b * 4 < nwords; ++b) {
        uint32_t ctr[4] = { call, (uint32_t)b, field, o->request }, out[4];
        or_philox4x32_10(ctr, o->key, out);
        for (int l = 0; l < 4 && 4 * b + l < nwords; ++l) X[4 * b + l] = out[l];
    }
}

/* R10: uniform in (0,1), never 0 or 1. */
static double unif(uint32_t X) { return ((double)X + 0.5) * 0x1p-32; }

/* ------------------------------------------------------------------ */
/* Grid rows.                                                          */
/* ------------------------------------------------------------------ */
static double *edge_row(const or_ctx *o, int c, int k) { return o->edges + ((size_t)c * o->d + k) * (o->n + 1); }

/* Eq. 12 / 26: the one-dimensional density of bin j is 1/(n Δx_j). */
static double bin_density(const or_ctx *o, const double *e, int j)
{
    return 1.0 / ((double)o->n * (e[j + 1] - e[j]));
}

/* R11: largest j in [0, n-1] with ξ_j <= x. */
static int bin_search(const double *e, int n, double x)
{
    int lo = 0, hi = n - 1; /* answer in [lo, hi] */
    if (!(x >= e[0])) return 0;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (e[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* ------------------------------------------------------------------ */
/* Channel maps φ_c (§3.4, §3.5): identity on unmapped coordinates.    */
/* ------------------------------------------------------------------ */
/* Forward: x_c -> p, and the density factor 1/φ'_c (product over slots). */
static void chan_forward(const or_maps *m, int d, const double *x, double *p, double *jac)
{
    for (int k = 0; k < d; ++k) p[k] = x[k];
    double J = 1.0;
    for (int s = 0; s < m->nmap; ++s) {
        int k = m->coord[s];
        if (m->kind[s] == OR_MAP_BW) {
            double mass = m->a[s], G = m->b[s], A = m->bwA[s];
            p[k] = mass + G * tan(A * x[k] - m->bwT0[s]);
            double dp = p[k] - mass;
            J *= G / (A * (dp * dp + G * G));
        } else if (m->kind[s] == OR_MAP_POW) {
            double x2 = x[k] * x[k], x4 = x2 * x2;
            double pk = x4 * x[k];
            if (pk < DBL_MIN) pk = DBL_MIN; /* R15 */
            p[k] = pk;
            J *= 1.0 / (5.0 * x4);
        }
    }
    *jac = J;
}

/* Inverse: p -> x_c = φ_c^{-1}(p) (R7), and 1/φ'_c at that point. */
static void chan_inverse(const or_maps *m, int d, const double *p, double *x, double *jac)
{
    for (int k = 0; k < d; ++k) x[k] = p[k];
    double J = 1.0;
    for (int s = 0; s < m->nmap; ++s) {
        int k = m->coord[s];
        if (m->kind[s] == OR_MAP_BW) {
            double mass = m->a[s], G = m->b[s], A = m->bwA[s];
            double dp = p[k] - mass;
            x[k] = (atan(dp / G) + m->bwT0[s]) / A;
            J *= G / (A * (dp * dp + G * G));
        } else if (m->kind[s] == OR_MAP_POW) {
            double xx = pow(p[k], 0.2);
            x[k] = xx;
            double x2 = xx * xx;
            J *= 1.0 / (5.0 * (x2 * x2));
        }
    }
    *jac = J;
}

/* ------------------------------------------------------------------ */
/* Synthetic integrand f(p) (stand-in for the matrix element, §3.1).   */
/* ------------------------------------------------------------------ */
static double gauss_factor(const or_ctx *o, double p)
{
    if (o->gsig == 0.0) return 1.0;
    double u = (p - o->gcen) / o->gsig;
    return exp(-0.5 * u * u) / o->gZ;
}

static double peak_factor(const or_maps *m, int s, double p)
{
    if (m->kind[s] == OR_MAP_BW) {
        double mass = m->a[s], G = m->b[s];
        double dp = p - mass;
        return G / (m->bwA[s] * (dp * dp + G * G));
    }
    if (m->kind[s] == OR_MAP_POW) {
        return pow(p + m->b[s], -0.8) / m->powN[s];
    }
    return 1.0;
}

double or_f(const or_ctx *o, const double *p)
{
    double f = 0.0;
    for (int q = 0; q < o->P; ++q) {
        const or_maps *m = &o->pk[q];
        double v = 1.0;
        for (int k = 0; k < o->d; ++k) {
            int s = m->slot_of[k];
            v *= (s >= 0) ? peak_factor(m, s, p[k]) : gauss_factor(o, p[k]);
        }
        f += o->pk_w[q] * v;
    }
    return f;
}

/* ------------------------------------------------------------------ */
/* Multi-channel density g(p), Eq. 30.                                 */
/* ------------------------------------------------------------------ */
/* g_c(x) = prod_k 1/(n Δx_{c,k,j_k}) for a channel's own grid (Eq. 26). */
static double grid_density(const or_ctx *o, int c, const double *x, int *bins)
{
    double g = 1.0;
    for (int k = 0; k < o->d; ++k) {
        const double *e = edge_row(o, c, k);
        int j = bin_search(e, o->n, x[k]);
        if (bins) bins[k] = j;
        g *= bin_density(o, e, j);
    }
    return g;
}

/* Sum over all channels c' of α_c' g_c'(x_c') / φ'_c'(x_c'), x_c' = φ_c'^{-1}(p).
 * For the channel that generated the point (own >= 0) the forward grid
 * value and Jacobian are used (no inversion, §3.5 work order). */
static double g_of_p(const or_ctx *o, int own, const double *p, double g_own, double jac_own,
                     const int *j_own, int *bins_all)
{
    double g = 0.0;
    double xq[OR_MAX_D];
    for (int c = 0; c < o->K; ++c) {
        if (o->alpha[c] == 0.0) {
            if (bins_all) for (int k = 0; k < o->d; ++k) bins_all[c * o->d + k] = -1;
            continue;
        }
        double term;
        if (c == own) {
            if (bins_all) for (int k = 0; k < o->d; ++k) bins_all[c * o->d + k] = j_own[k];
            term = o->alpha[c] * g_own * jac_own;
        } else {
            double J;
            chan_inverse(&o->ch[c], o->d, p, xq, &J);
            double gc = grid_density(o, c, xq, bins_all ? bins_all + c * o->d : NULL);
            term = o->alpha[c] * gc * J;
        }
        g += term;
    }
    return g;
}

/* One call of channel c from its random words: §3.5 work order.
 * Returns w = f(p)/g(p); fills x (channel coordinates), p, forward bins. */
static double eval_call(const or_ctx *o, int c, const uint32_t *X, const int64_t *digit, int64_t nr,
                        double *x, double *p, int *jf, int *bins_all, double *f_out, double *g_out)
{
    const double *e;
    double gc = 1.0;
    /* x_c = G_c^{-1}(r): bin index and in-bin fraction from the integer
     * (2X+1) n (R10), or (2^33 a_k + 2X + 1) n over n_r 2^33 in a
     * stratification cell with digits a_k (R16); linear inside the bin (§3.2). */
    for (int k = 0; k < o->d; ++k) {
        int j;
        double fr;
        if (digit) {
            const uint64_t den = (uint64_t)nr << 33;
            const uint64_t t = (((uint64_t)digit[k] << 33) + 2ull * X[k] + 1ull) * (uint64_t)o->n;
            j = (int)(t / den);
            fr = (double)(t % den) / (double)den;
        } else {
            uint64_t t = (2ull * X[k] + 1ull) * (uint64_t)o->n;
            j = (int)(t >> 33);
            fr = (double)(t & ((1ull << 33) - 1ull)) * 0x1p-33;
        }
        e = edge_row(o, c, k);
        double w = e[j + 1] - e[j];
        x[k] = e[j] + fr * w;
        jf[k] = j;
        gc *= bin_density(o, e, j);
    }
    double jac;
    chan_forward(&o->ch[c], o->d, x, p, &jac);
    double f = or_f(o, p);
    double g = g_of_p(o, c, p, gc, jac, jf, bins_all);
    if (f_out) *f_out = f;
    if (g_out) *g_out = g;
    if (!(g > 0.0)) return 0.0;
    return f / g;
}

/* ------------------------------------------------------------------ */
/* Context.                                                            */
/* ------------------------------------------------------------------ */
static int load_maps(or_maps *dst, int cnt, int d, const int32_t *nmap, const int32_t *coord,
                     const int32_t *kind, const double *a, const double *b)
{
    for (int q = 0; q < cnt; ++q) {
        or_maps *m = &dst[q];
        memset(m, 0, sizeof *m);
        for (int k = 0; k < OR_MAX_D; ++k) m->slot_of[k] = -1;
        m->nmap = nmap[q];
        if (m->nmap < 0 || m->nmap > OR_MAX_MAPPED) return OR_ERR_ARG;
        for (int s = 0; s < m->nmap; ++s) {
            m->coord[s] = coord[q * 4 + s];
            m->kind[s] = kind[q * 4 + s];
            m->a[s] = a[q * 4 + s];
            m->b[s] = b[q * 4 + s];
            int k = m->coord[s];
            if (k < 0 || k >= d || m->slot_of[k] >= 0) return OR_ERR_ARG;
            m->slot_of[k] = s;
            if (m->kind[s] == OR_MAP_BW) {
                double mass = m->a[s], G = m->b[s];
                if (!(G > 0.0)) return OR_ERR_ARG;
                /* ∫_0^1 Γ/((p-m)²+Γ²) dp */
                m->bwA[s] = atan((1.0 - mass) / G) + atan(mass / G);
                m->bwT0[s] = atan(mass / G);
            } else if (m->kind[s] == OR_MAP_POW) {
                double del = m->b[s];
                if (!(del >= 0.0)) return OR_ERR_ARG;
                /* ∫_0^1 (p+δ)^-0.8 dp */
                m->powN[s] = 5.0 * (pow(1.0 + del, 0.2) - pow(del, 0.2));
            } else if (m->kind[s] != OR_MAP_ID) {
                return OR_ERR_ARG;
            }
        }
    }
    return OR_OK;
}

void or_destroy(or_ctx *o)
{
    if (!o) return;
    free(o->ch); free(o->pk); free(o->pk_w); free(o->edges); free(o->alpha); free(o->shift);
    free(o->Nc); free(o->Pc); free(o->D); free(o->Ic); free(o->Vc); free(o->Wc);
    free(o->nr); free(o->spc); free(o->Cc);
    free(o->eq); free(o->Dp);
    free(o);
}

or_ctx *or_create(const or_problem *pr, int *status)
{
    *status = OR_ERR_ARG;
    if (pr->d < 1 || pr->d > OR_MAX_D || pr->n_channels < 1 || pr->n_bins < 1 || pr->n_peaks < 1)
        return NULL;
    or_ctx *o = calloc(1, sizeof *o);
    if (!o) { *status = OR_ERR_MEM; return NULL; }
    o->d = pr->d; o->K = pr->n_channels; o->n = pr->n_bins; o->P = pr->n_peaks;
    o->ch = calloc(o->K, sizeof(or_maps));
    o->pk = calloc(o->P, sizeof(or_maps));
    o->pk_w = calloc(o->P, sizeof(double));
    size_t ne = (size_t)o->K * o->d * (o->n + 1), nd = (size_t)o->K * o->d * o->n;
    o->edges = calloc(ne, sizeof(double));
    o->D = calloc(nd, sizeof(double));
    o->alpha = calloc(o->K, sizeof(double));
    o->shift = calloc(o->K, sizeof(double));
    o->Nc = calloc(o->K, sizeof(int64_t));
    o->Pc = calloc(o->K + 1, sizeof(int64_t));
    o->Ic = calloc(o->K, sizeof(double));
    o->Vc = calloc(o->K, sizeof(double));
    o->Wc = calloc(o->K, sizeof(double));
    o->nr = calloc(o->K, sizeof(int64_t));
    o->spc = calloc(o->K, sizeof(int64_t));
    o->Cc = calloc(o->K, sizeof(int64_t));
    if (!o->ch || !o->pk || !o->pk_w || !o->edges || !o->D || !o->alpha || !o->shift || !o->Nc ||
        !o->Pc || !o->Ic || !o->Vc || !o->Wc || !o->nr || !o->spc || !o->Cc) {
        or_destroy(o); *status = OR_ERR_MEM; return NULL;
    }
    o->stratified = pr->stratified ? 1 : 0;
    if (pr->n_equiv < 0 || (pr->n_equiv > 0 && !pr->equiv)) { or_destroy(o); return NULL; }
    if (pr->n_equiv > 0) {
        const int rl = 2 + 2 * o->d;
        o->n_eq = pr->n_equiv;
        o->eq = malloc((size_t)o->n_eq * rl * sizeof(int32_t));
        o->Dp = calloc(nd, sizeof(double));
        if (!o->eq || !o->Dp) { or_destroy(o); *status = OR_ERR_MEM; return NULL; }
        memcpy(o->eq, pr->equiv, (size_t)o->n_eq * rl * sizeof(int32_t));
        for (int e = 0; e < o->n_eq; ++e) {
            const int32_t *r = o->eq + (size_t)e * rl;
            int bad = r[0] < 0 || r[0] >= o->K || r[1] < 0 || r[1] >= o->K;
            for (int k = 0; k < o->d && !bad; ++k) {
                bad = r[2 + k] < 0 || r[2 + k] >= o->d || r[2 + o->d + k] < 0 || r[2 + o->d + k] > 3;
                for (int q = 0; q < k && !bad; ++q) bad = r[2 + q] == r[2 + k]; /* π a permutation */
            }
            if (bad) { or_destroy(o); return NULL; }
        }
    }
    if (load_maps(o->ch, o->K, o->d, pr->ch_nmap, pr->ch_coord, pr->ch_kind, pr->ch_a, pr->ch_b) ||
        load_maps(o->pk, o->P, o->d, pr->pk_nmap, pr->pk_coord, pr->pk_kind, pr->pk_a, pr->pk_b)) {
        or_destroy(o); return NULL;
    }
    memcpy(o->pk_w, pr->pk_w, o->P * sizeof(double));
    o->gsig = pr->gauss_sigma; o->gcen = pr->gauss_centre; o->gnorm = pr->gauss_norm;
    if (o->gsig < 0.0) { or_destroy(o); return NULL; }
    if (o->gsig > 0.0) {
        if (o->gnorm == 0) o->gZ = o->gsig * sqrt(2.0 * M_PI);
        else o->gZ = o->gsig * sqrt(M_PI / 2.0) *
                     (erf((1.0 - o->gcen) / (o->gsig * M_SQRT2)) + erf(o->gcen / (o->gsig * M_SQRT2)));
    }
    o->key[0] = (uint32_t)(pr->seed & 0xffffffffu);
    o->key[1] = (uint32_t)(pr->seed >> 32);
    o->request = pr->request_id;
    o->grid_alpha = pr->grid_alpha; o->beta = pr->beta; o->n_min = pr->n_min;
    o->smooth = pr->smooth; o->omega_mode = pr->omega_mode;
    o->gen_batch = pr->gen_batch > 0 ? pr->gen_batch : (1 << 20);
    /* Initial state: equidistant bins, α_c = 1/K (§3.4, §3.5). */
    for (int c = 0; c < o->K; ++c) {
        o->alpha[c] = 1.0 / (double)o->K;
        for (int k = 0; k < o->d; ++k) {
            double *e = edge_row(o, c, k);
            for (int j = 0; j <= o->n; ++j) e[j] = (double)j / (double)o->n;
        }
    }
    *status = OR_OK;
    return o;
}

/* ------------------------------------------------------------------ */
/* Call allocation, R6 (§3.4: integer N_c with a lower threshold).     */
/* ------------------------------------------------------------------ */
int64_t or_allocate_raw(int K, const double *alpha, int64_t N, int64_t n_min, int64_t *Nc, int64_t *Pc)
{
    Pc[0] = 0;
    for (int c = 0; c < K; ++c) {
        int64_t nc = 0;
        if (alpha[c] > 0.0) {
            nc = (int64_t)floor(alpha[c] * (double)N);
            if (nc < n_min) nc = n_min;
        }
        Nc[c] = nc;
        Pc[c + 1] = Pc[c] + nc;
    }
    return Pc[K];
}

/* R16: the largest m in [1, 2^20] with 2 m^d <= N (1 if N < 2^(d+1)). */
int64_t or_strat_cells_per_axis(int64_t N, int d)
{
    int64_t lo = 1, hi = 1 << 20;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2, prod = 2;
        for (int k = 0; k < d && prod <= N; ++k) {
            if (prod > N / mid) { prod = N + 1; break; }
            prod *= mid;
        }
        if (prod <= N) lo = mid; else hi = mid - 1;
    }
    return lo;
}

int64_t or_allocate(or_ctx *o, int64_t N)
{
    o->n_total = or_allocate_raw(o->K, o->alpha, N, o->n_min, o->Nc, o->Pc);
    if (o->stratified) {
        o->Pc[0] = 0;
        for (int c = 0; c < o->K; ++c) {
            int64_t m = 1, C = 1, s = o->Nc[c];
            if (o->Nc[c] >= 2) {
                m = or_strat_cells_per_axis(o->Nc[c], o->d);
                C = 1;
                for (int k = 0; k < o->d; ++k) C *= m;
                s = o->Nc[c] / C;
            }
            o->nr[c] = m; o->Cc[c] = C; o->spc[c] = s;
            o->Nc[c] = s * C;
            o->Pc[c + 1] = o->Pc[c] + o->Nc[c];
        }
        o->n_total = o->Pc[o->K];
    }
    return o->n_total;
}

/* ------------------------------------------------------------------ */
/* Sampling pass (Eqs. 10, 11, 15, 23, 31).                            */
/* ------------------------------------------------------------------ */
typedef struct {
    const or_ctx *o;
    uint32_t iteration;
    int64_t i0, i1;           /* calls (importance) or cells (stratified) */
    const int64_t *cell_off;  /* K+1: first cell of each channel (stratified) */
    ksum *S1, *S2, *D, *Q;    /* Q: Σ_cells (Σ_cell d)^2 per channel (R17) */
    double wmax;
    int bad;
} pass_part;

/* One call: weight, shifted sums, d-values, w_max. */
static double pass_call(pass_part *pp, int c, int64_t i, const int64_t *digit, uint32_t *X, double *x,
                        double *p, int *jf)
{
    const or_ctx *o = pp->o;
    const int d = o->d, n = o->n;
    call_words(o, (uint32_t)i, pp->iteration, d, X);
    double w = eval_call(o, c, X, digit, digit ? o->nr[c] : 0, x, p, jf, NULL, NULL, NULL);
    if (!isfinite(w)) { pp->bad = 1; w = 0.0; }
    double dv = w - o->shift[c];
    ks_add(&pp->S1[c], dv);
    ks_add(&pp->S2[c], dv * dv);
    double w2 = w * w;
    for (int k = 0; k < d; ++k) ks_add(&pp->D[((size_t)c * d + k) * n + jf[k]], w2);
    if (fabs(w) > pp->wmax) pp->wmax = fabs(w); /* R19 */
    return dv;
}

static void *pass_worker(void *arg)
{
    pass_part *pp = arg;
    const or_ctx *o = pp->o;
    uint32_t X[OR_MAX_D + 4];
    double x[OR_MAX_D], p[OR_MAX_D];
    int jf[OR_MAX_D];
    int c = 0;
    if (!o->stratified) {
        while (c < o->K && o->Pc[c + 1] <= pp->i0) ++c;
        for (int64_t i = pp->i0; i < pp->i1; ++i) {
            while (o->Pc[c + 1] <= i) ++c;
            pass_call(pp, c, i, NULL, X, x, p, jf);
        }
        return NULL;
    }
    /* R16/R17: whole cells; the s calls of a cell are consecutive */
    int64_t digit[OR_MAX_D];
    while (c < o->K && pp->cell_off[c + 1] <= pp->i0) ++c;
    for (int64_t q = pp->i0; q < pp->i1; ++q) {
        while (pp->cell_off[c + 1] <= q) ++c;
        const int64_t l = q - pp->cell_off[c];
        int64_t rest = l;
        for (int k = 0; k < o->d; ++k) { digit[k] = rest % o->nr[c]; rest /= o->nr[c]; }
        ksum cs = {0, 0};
        for (int64_t m = 0; m < o->spc[c]; ++m)
            ks_add(&cs, pass_call(pp, c, o->Pc[c] + l * o->spc[c] + m, digit, X, x, p, jf));
        const double v = ks_val(&cs);
        ks_add(&pp->Q[c], v * v);
    }
    return NULL;
}

static void combine_history(or_ctx *o)
{
    /* R9: inverse-variance weighted mean of the flagged passes. */
    int cnt = 0, nzero = 0;
    ksum zI = {0, 0};
    for (int h = 0; h < o->n_hist; ++h) {
        if (!o->hist_comb[h]) continue;
        ++cnt;
        if (o->hist_V[h] <= 0.0) { ++nzero; ks_add(&zI, o->hist_I[h]); }
    }
    o->comb_I = 0.0; o->comb_sigma = 0.0; o->comb_chi2 = 0.0;
    if (cnt == 0) return;
    if (nzero > 0) { o->comb_I = ks_val(&zI) / nzero; return; }
    ksum sw = {0, 0}, swi = {0, 0};
    for (int h = 0; h < o->n_hist; ++h) {
        if (!o->hist_comb[h]) continue;
        ks_add(&sw, 1.0 / o->hist_V[h]);
        ks_add(&swi, o->hist_I[h] / o->hist_V[h]);
    }
    double Ibar = ks_val(&swi) / ks_val(&sw);
    o->comb_I = Ibar;
    o->comb_sigma = sqrt(1.0 / ks_val(&sw));
    if (cnt > 1) {
        ksum chi = {0, 0};
        for (int h = 0; h < o->n_hist; ++h) {
            if (!o->hist_comb[h]) continue;
            double dI = o->hist_I[h] - Ibar;
            ks_add(&chi, dI * dI / o->hist_V[h]);
        }
        o->comb_chi2 = ks_val(&chi) / (double)(cnt - 1);
    }
}

/* out[0..7] = integral, variance, w_max, efficiency, n_calls, combined,
 * combined_sigma, chi2_dof. */
int or_sample_pass(or_ctx *o, int64_t N, uint32_t iteration, int combine, int n_threads, double *out)
{
    if (N < 1 || iteration >= 0x80000000u) return OR_ERR_ARG;
    int64_t Nt = or_allocate(o, N);
    if (Nt > 0xffffffffll) return OR_ERR_ARG;
    int K = o->K, d = o->d, n = o->n;
    size_t nd = (size_t)K * d * n;
    if (n_threads < 1) n_threads = 1;
    if ((int64_t)n_threads > Nt) n_threads = (int)(Nt > 0 ? Nt : 1);
    pass_part *parts = calloc(n_threads, sizeof *parts);
    pthread_t *th = calloc(n_threads, sizeof *th);
    int64_t *cell_off = calloc(K + 1, sizeof(int64_t));
    for (int c = 0; c < K; ++c) cell_off[c + 1] = cell_off[c] + (o->stratified ? o->Cc[c] : 0);
    const int64_t units = o->stratified ? cell_off[K] : Nt;  /* split by cells when stratified */
    int rc = OR_OK;
    for (int t = 0; t < n_threads; ++t) {
        parts[t].o = o;
        parts[t].iteration = iteration;
        parts[t].i0 = units * t / n_threads;
        parts[t].i1 = units * (t + 1) / n_threads;
        parts[t].cell_off = cell_off;
        parts[t].S1 = calloc(K, sizeof(ksum));
        parts[t].S2 = calloc(K, sizeof(ksum));
        parts[t].Q = calloc(K, sizeof(ksum));
        parts[t].D = calloc(nd, sizeof(ksum));
        parts[t].wmax = 0.0;
        if (!parts[t].S1 || !parts[t].S2 || !parts[t].Q || !parts[t].D) rc = OR_ERR_MEM;
    }
    if (rc == OR_OK) {
        if (n_threads == 1) pass_worker(&parts[0]);
        else {
            for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, pass_worker, &parts[t]);
            for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
        }
        /* ordered merge of the partial compensated sums */
        double wmax = 0.0;
        int bad = 0;
        for (int c = 0; c < K; ++c) {
            ksum s1 = {0, 0}, s2 = {0, 0}, qq = {0, 0};
            for (int t = 0; t < n_threads; ++t) {
                ks_add(&s1, parts[t].S1[c].s); ks_add(&s1, parts[t].S1[c].c);
                ks_add(&s2, parts[t].S2[c].s); ks_add(&s2, parts[t].S2[c].c);
                ks_add(&qq, parts[t].Q[c].s); ks_add(&qq, parts[t].Q[c].c);
            }
            double Nc = (double)o->Nc[c];
            if (o->Nc[c] == 0) { o->Ic[c] = o->Vc[c] = o->Wc[c] = 0.0; continue; }
            double m1 = ks_val(&s1) / Nc, m2 = ks_val(&s2) / Nc;
            /* Eqs. 10, 11 per channel, on sums shifted by s_c (R13). */
            o->Ic[c] = o->shift[c] + m1;
            double V = 0.0;
            if (!o->stratified) {
                if (o->Nc[c] > 1) V = (m2 - m1 * m1) * Nc / (Nc - 1.0);
            } else if (o->spc[c] >= 2) {
                /* R17: mean over cells of the cell sample variances */
                const double s = (double)o->spc[c];
                V = (ks_val(&s2) - ks_val(&qq) / s) / ((double)o->Cc[c] * (s - 1.0));
            }
            if (V < 0.0) V = 0.0;
            o->Vc[c] = V;
            o->Wc[c] = (m2 - m1 * m1) + o->Ic[c] * o->Ic[c];
        }
        for (size_t q = 0; q < nd; ++q) {
            ksum s = {0, 0};
            for (int t = 0; t < n_threads; ++t) { ks_add(&s, parts[t].D[q].s); ks_add(&s, parts[t].D[q].c); }
            o->D[q] = ks_val(&s);
        }
        for (int t = 0; t < n_threads; ++t) {
            if (parts[t].wmax > wmax) wmax = parts[t].wmax;
            bad |= parts[t].bad;
        }
        /* Eq. 23 (general α form) and R8. */
        ksum I = {0, 0}, V = {0, 0};
        for (int c = 0; c < K; ++c) {
            if (o->Nc[c] == 0) continue;
            ks_add(&I, o->alpha[c] * o->Ic[c]);
            ks_add(&V, o->alpha[c] * o->alpha[c] * o->Vc[c] / (double)o->Nc[c]);
        }
        for (int c = 0; c < K; ++c) o->shift[c] = o->Ic[c];
        o->wmax = wmax;
        o->have_pass = 1;
        if (o->n_hist < OR_MAX_HIST) {
            o->hist_I[o->n_hist] = ks_val(&I);
            o->hist_V[o->n_hist] = ks_val(&V);
            o->hist_comb[o->n_hist] = combine ? 1 : 0;
            o->n_hist++;
        }
        combine_history(o);
        out[0] = ks_val(&I);
        out[1] = ks_val(&V);
        out[2] = wmax;
        out[3] = wmax > 0.0 ? ks_val(&I) / wmax : 0.0; /* Eq. 2 */
        out[4] = (double)Nt;
        out[5] = o->comb_I;
        out[6] = o->comb_sigma;
        out[7] = o->comb_chi2;
        if (bad) rc = OR_ERR_NUMERIC;
    }
    for (int t = 0; t < n_threads; ++t) {
        free(parts[t].S1); free(parts[t].S2); free(parts[t].Q); free(parts[t].D);
    }
    free(parts); free(th); free(cell_off);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Grid refinement, Eqs. 14, 15 with R1-R4.                            */
/* ------------------------------------------------------------------ */
static void refine_row(const double *Din, int n, int smooth, double alpha_grid, double *e)
{
    double *Dj = malloc(n * sizeof(double)), *m = malloc(n * sizeof(double));
    double *C = malloc((n + 1) * sizeof(double)), *ne = malloc((n + 1) * sizeof(double));
    for (int j = 0; j < n; ++j) Dj[j] = Din[j];
    if (smooth && n >= 2) { /* R3 */
        double *t = malloc(n * sizeof(double));
        t[0] = (Din[0] + Din[1]) / 2.0;
        t[n - 1] = (Din[n - 2] + Din[n - 1]) / 2.0;
        for (int j = 1; j < n - 1; ++j) t[j] = (Din[j - 1] + Din[j] + Din[j + 1]) / 3.0;
        for (int j = 0; j < n; ++j) Dj[j] = t[j];
        free(t);
    }
    /* ω_j = sqrt(Σ w²) of the bin (Eq. 15); r_j = ω_j / Σ ω. */
    double S = 0.0;
    for (int j = 0; j < n; ++j) { Dj[j] = sqrt(Dj[j]); S += Dj[j]; }
    if (S > 0.0) {
        for (int j = 0; j < n; ++j) {
            double r = Dj[j] / S;
            double mj;
            if (r == 0.0) mj = 0.0;                    /* R2 */
            else if (fabs(r - 1.0) < 1e-12) mj = 1.0;   /* R2 */
            else mj = pow((r - 1.0) / log(r), alpha_grid); /* Eq. 14 */
            m[j] = mj;
        }
        C[0] = 0.0;
        for (int j = 0; j < n; ++j) C[j + 1] = C[j] + m[j];
        double M = C[n];
        if (M > 0.0) {
            /* R4: new edge i sits where the cumulative of m, linear inside
             * each old bin, reaches i M / n. */
            ne[0] = 0.0;
            ne[n] = 1.0;
            int j = 1;
            for (int i = 1; i < n; ++i) {
                double t = (double)i * M / (double)n;
                while (j < n && C[j] < t) ++j;
                /* C_{j-1} < t <= C_j, old bin j-1 = [e_{j-1}, e_j] */
                double fr = (t - C[j - 1]) / m[j - 1];
                ne[i] = e[j - 1] + fr * (e[j] - e[j - 1]);
            }
            for (int i = 0; i <= n; ++i) e[i] = ne[i];
        }
    }
    free(Dj); free(m); free(C); free(ne);
}

/* R18: bin weights of every channel after the channel equivalences. */
static void pool_equivalences(or_ctx *o)
{
    const int d = o->d, n = o->n, rl = 2 + 2 * d;
    for (int c = 0; c < o->K; ++c)
        for (int k = 0; k < d; ++k) {
            double *out = o->Dp + ((size_t)c * d + k) * n;
            const double *own = o->D + ((size_t)c * d + k) * n;
            int invariant = 0;
            for (int j = 0; j < n; ++j) out[j] = own[j];
            for (int e = 0; e < o->n_eq; ++e) {
                const int32_t *r = o->eq + (size_t)e * rl;
                if (r[0] != c) continue;
                const int mode = r[2 + d + k];
                const double *src = o->D + ((size_t)r[1] * d + r[2 + k]) * n;
                for (int j = 0; j < n; ++j) {
                    if (mode == OR_EQ_IDENTITY) out[j] += src[j];
                    else if (mode == OR_EQ_INVERT) out[j] += src[n - 1 - j];
                    else if (mode == OR_EQ_SYMMETRIC) out[j] += 0.5 * (src[j] + src[n - 1 - j]);
                }
                if (mode == OR_EQ_INVARIANT) invariant = 1;
            }
            if (invariant)
                for (int j = 0; j < n; ++j) out[j] = 1.0;
        }
}

int or_refine_grids(or_ctx *o)
{
    if (!o->have_pass) return OR_ERR_STATE;
    const double *W = o->D;
    if (o->n_eq > 0) { pool_equivalences(o); W = o->Dp; }
    for (int c = 0; c < o->K; ++c)
        for (int k = 0; k < o->d; ++k)
            refine_row(W + ((size_t)c * o->d + k) * o->n, o->n, o->smooth, o->grid_alpha,
                       edge_row(o, c, k));
    return OR_OK;
}

/* The bin weights the next refinement would use (R18; D itself without
 * equivalences). */
int or_get_pooled(or_ctx *o, double *out)
{
    if (!o->have_pass) return OR_ERR_STATE;
    const size_t nd = (size_t)o->K * o->d * o->n;
    if (o->n_eq > 0) { pool_equivalences(o); memcpy(out, o->Dp, nd * sizeof(double)); }
    else memcpy(out, o->D, nd * sizeof(double));
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Channel-weight update, Eq. 25 with R5.                              */
/* ------------------------------------------------------------------ */
/* Pure form of the update: alpha_out from alpha, ω_c, I_c and N_c. */
void or_alpha_update_raw(int K, const double *alpha, const double *omega, const double *Ic,
                         const int64_t *Nc, double beta, double *alpha_out)
{
    double SU = 0.0, MU = 0.0;
    for (int c = 0; c < K; ++c) {
        if (alpha[c] > 0.0 && Nc[c] > 0 && omega[c] > 0.0) {
            SU += alpha[c] * pow(omega[c], beta);
            MU += alpha[c];
        }
    }
    double tot = 0.0;
    for (int c = 0; c < K; ++c) {
        double a = alpha[c];
        if (a > 0.0 && Nc[c] > 0) {
            if (omega[c] > 0.0) a = alpha[c] * pow(omega[c], beta) / SU * MU; /* Eq. 25 */
            else if (Ic[c] == 0.0) a = 0.0; /* all calls gave w = 0: switch off */
            /* else: no variance information, α_c kept */
        }
        alpha_out[c] = a;
        tot += a;
    }
    if (tot > 0.0) for (int c = 0; c < K; ++c) alpha_out[c] /= tot;
    else for (int c = 0; c < K; ++c) alpha_out[c] = alpha[c];
}

int or_update_alpha(or_ctx *o)
{
    if (!o->have_pass) return OR_ERR_STATE;
    double *om = malloc(o->K * sizeof(double)), *na = malloc(o->K * sizeof(double));
    for (int c = 0; c < o->K; ++c) om[c] = o->omega_mode ? o->Wc[c] : o->Vc[c];
    or_alpha_update_raw(o->K, o->alpha, om, o->Ic, o->Nc, o->beta, na);
    memcpy(o->alpha, na, o->K * sizeof(double));
    free(om); free(na);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Unweighted event generation (§2 Eq. 2, §3.3, §3.5) with R12.        */
/* ------------------------------------------------------------------ */
static int choose_channel(const or_ctx *o, const double *A, double u)
{
    double tgt = u * A[o->K - 1];
    for (int c = 0; c < o->K; ++c)
        if (tgt < A[c]) return c;
    for (int c = o->K - 1; c >= 0; --c)
        if (o->alpha[c] > 0.0) return c;
    return 0;
}

int or_generate(or_ctx *o, int64_t n_events, uint32_t gen_id, float *p_out, double *w_out,
                int64_t *stats /* n_written, n_calls_used, n_overweight, n_batches */)
{
    if (!o->have_pass) return OR_ERR_STATE;
    if (n_events < 0 || gen_id >= 0x8000u) return OR_ERR_ARG;
    int d = o->d, K = o->K;
    double *A = malloc(K * sizeof(double));
    double acc = 0.0;
    for (int c = 0; c < K; ++c) { acc += o->alpha[c]; A[c] = acc; }
    uint32_t X[OR_MAX_D + 4];
    double x[OR_MAX_D], p[OR_MAX_D];
    int jf[OR_MAX_D];
    int64_t written = 0, used = 0, over = 0, b = 0;
    int rc = OR_OK;
    while (written < n_events) {
        if (b >= 0x10000) { rc = OR_ERR_NUMERIC; break; }
        uint32_t field = 0x80000000u | (gen_id << 16) | (uint32_t)b;
        double bmax = 0.0;
        double wm = o->wmax;
        for (int64_t i = 0; i < o->gen_batch; ++i) {
            call_words(o, (uint32_t)i, field, d + 2, X);
            int c = choose_channel(o, A, unif(X[d]));
            double w = eval_call(o, c, X, NULL, 0, x, p, jf, NULL, NULL, NULL);
            if (!isfinite(w)) { rc = OR_ERR_NUMERIC; w = 0.0; }
            if (fabs(w) > bmax) bmax = fabs(w);
            if (written < n_events) {
                ++used;
                if (unif(X[d + 1]) * wm < fabs(w)) { /* R19: keep the sign */
                    for (int k = 0; k < d; ++k) p_out[written * d + k] = (float)p[k];
                    w_out[written] = w;
                    if (fabs(w) > wm) ++over;
                    ++written;
                }
            }
        }
        if (bmax > o->wmax) o->wmax = bmax;
        ++b;
    }
    stats[0] = written; stats[1] = used; stats[2] = over; stats[3] = b;
    free(A);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Diagnostics for parity tests.                                       */
/* ------------------------------------------------------------------ */
/* mode 0: integration call `call` of pass `field` (channel from the last
 * allocation); mode 1: generation call (channel drawn from α).
 * out_d[0..3] = f, g, w, channel; x, p: d values; bins: K*d (-1 = skipped). */
int or_eval_call(const or_ctx *o, int mode, uint32_t field, uint32_t call, double *x, double *p,
                 int32_t *jf, int32_t *bins_all, uint32_t *words, double *out_d)
{
    uint32_t X[OR_MAX_D + 4];
    int d = o->d;
    int c;
    int jfi[OR_MAX_D];
    int *ball = NULL;
    if (bins_all) ball = malloc((size_t)o->K * d * sizeof(int));
    int64_t digit[OR_MAX_D];
    int strat = 0;
    if (mode == 0) {
        if ((int64_t)call >= o->n_total) { free(ball); return OR_ERR_ARG; }
        c = 0;
        while (o->Pc[c + 1] <= (int64_t)call) ++c;
        call_words(o, call, field, d, X);
        if (words) for (int k = 0; k < d; ++k) words[k] = X[k];
        if (o->stratified) {
            int64_t rest = ((int64_t)call - o->Pc[c]) / o->spc[c];
            for (int k = 0; k < d; ++k) { digit[k] = rest % o->nr[c]; rest /= o->nr[c]; }
            strat = 1;
        }
    } else {
        double *A = malloc(o->K * sizeof(double));
        double acc = 0.0;
        for (int q = 0; q < o->K; ++q) { acc += o->alpha[q]; A[q] = acc; }
        call_words(o, call, field, d + 2, X);
        if (words) for (int k = 0; k < d + 2; ++k) words[k] = X[k];
        c = choose_channel(o, A, unif(X[d]));
        free(A);
    }
    double f, g;
    double w = eval_call(o, c, X, strat ? digit : NULL, strat ? o->nr[c] : 0, x, p, jfi, ball, &f, &g);
    for (int k = 0; k < d; ++k) jf[k] = jfi[k];
    if (bins_all) for (int q = 0; q < o->K * d; ++q) bins_all[q] = ball[q];
    free(ball);
    out_d[0] = f; out_d[1] = g; out_d[2] = w; out_d[3] = (double)c;
    return OR_OK;
}

/* g(p) with every channel inverted (no own channel): Eq. 30 as a function. */
double or_g_point(const or_ctx *o, const double *p)
{
    return g_of_p(o, -1, p, 0.0, 0.0, NULL, NULL);
}

/* g_c(x) for one channel's grid (Eq. 26). */
double or_grid_density(const or_ctx *o, int c, const double *x)
{
    return grid_density(o, c, x, NULL);
}

/* Channel map and its inverse, exposed for round-trip tests. */
void or_channel_forward(const or_ctx *o, int c, const double *x, double *p, double *jac)
{
    chan_forward(&o->ch[c], o->d, x, p, jac);
}
void or_channel_inverse(const or_ctx *o, int c, const double *p, double *x, double *jac)
{
    chan_inverse(&o->ch[c], o->d, p, x, jac);
}

/* Refinement of one stand-alone row (for worked examples). */
void or_refine_row(const double *D, int n, int smooth, double alpha_grid, double *edges)
{
    refine_row(D, n, smooth, alpha_grid, edges);
}

/* State access (host arrays, caller-owned). */
void or_get_state(const or_ctx *o, double *edges, double *alpha, double *shift, double *wmax)
{
    size_t ne = (size_t)o->K * o->d * (o->n + 1);
    if (edges) memcpy(edges, o->edges, ne * sizeof(double));
    if (alpha) memcpy(alpha, o->alpha, o->K * sizeof(double));
    if (shift) memcpy(shift, o->shift, o->K * sizeof(double));
    if (wmax) *wmax = o->wmax;
}
void or_set_state(or_ctx *o, const double *edges, const double *alpha, const double *shift, double wmax,
                  int have_pass)
{
    size_t ne = (size_t)o->K * o->d * (o->n + 1);
    if (edges) memcpy(o->edges, edges, ne * sizeof(double));
    if (alpha) memcpy(o->alpha, alpha, o->K * sizeof(double));
    if (shift) memcpy(o->shift, shift, o->K * sizeof(double));
    o->wmax = wmax;
    o->have_pass = have_pass;
}
void or_get_pass(const or_ctx *o, double *D, double *Ic, double *Vc, int64_t *Nc)
{
    size_t nd = (size_t)o->K * o->d * o->n;
    if (D) memcpy(D, o->D, nd * sizeof(double));
    if (Ic) memcpy(Ic, o->Ic, o->K * sizeof(double));
    if (Vc) memcpy(Vc, o->Vc, o->K * sizeof(double));
    if (Nc) memcpy(Nc, o->Nc, o->K * sizeof(int64_t));
}

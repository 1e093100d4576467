"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, not by the oracle itself (CPU only).

Each test names the part of the method it pins; together they are chosen so
that a dropped term, a wrong sign, index or exponent, or a transposed
operand in any step of the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.stats as st
from numpy.polynomial.legendre import leggauss

from paper_1811_09711_gb300 import problems as P


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def two_channel_problem(seed=11, n_bins=10, d=2, width=3e-3, pow_second=False):
    """d=2 problem: peak/channel 0 = Breit-Wigner on coordinate 0, peak/channel
    1 = Breit-Wigner (or power law) on coordinate 1, Gaussian(0.2) elsewhere."""
    ms = P.MapSet.identity(2)
    ms.n_mapped[:] = 1
    ms.coord[0, 0], ms.kind[0, 0], ms.a[0, 0], ms.b[0, 0] = 0, P.MAP_BW, 0.37, width
    if pow_second:
        ms.coord[1, 0], ms.kind[1, 0], ms.a[1, 0], ms.b[1, 0] = 1, P.MAP_POW, 0.0, 2e-3
    else:
        ms.coord[1, 0], ms.kind[1, 0], ms.a[1, 0], ms.b[1, 0] = 1, P.MAP_BW, 0.61, 2 * width
    return P.Problem(name="two_channel", d=d, n_bins=n_bins, channels=ms,
                     peak_weight=np.array([0.6, 0.4]), peaks=ms.copy(), gauss_sigma=0.2,
                     gauss_centre=0.5, gauss_norm=P.GAUSS_NORM_UNIT, seed=seed,
                     iterations=4, calls=4000, adapt_grid=True, adapt_alpha=True)


def adapt(o, pr, iters, calls=None):
    last = None
    for it in range(iters):
        last = o.sample_pass(calls or pr.calls, it)
        o.refine_grids()
        if pr.adapt_alpha:
            o.update_alpha()
    return last


def bw_cdf(p, m, g):
    A = math.atan((1 - m) / g) + math.atan(m / g)
    return (np.arctan((p - m) / g) + math.atan(m / g)) / A


def tgauss_cdf(p, c=0.5, s=0.2):
    z = s * math.sqrt(2.0)
    lo, hi = math.erf(-c / z), math.erf((1 - c) / z)
    from scipy.special import erf
    return (erf((p - c) / z) - lo) / (hi - lo)


def pow_cdf(p, delta):
    return ((p + delta) ** 0.2 - delta ** 0.2) / ((1 + delta) ** 0.2 - delta ** 0.2)


def breakpoints_bw(m, g, n=160):
    """p-points that resolve a Breit-Wigner of mass m and width g."""
    A = math.atan((1 - m) / g) + math.atan(m / g)
    x = np.linspace(0.0, 1.0, n + 1)
    return m + g * np.tan(A * x - math.atan(m / g))


def gl_integrate_2d(fun, bx, by, order=8):
    """Tensor Gauss-Legendre quadrature over the cells of breakpoints bx, by."""
    xs, ws = leggauss(order)
    tot = 0.0
    bx = np.unique(np.clip(bx, 0, 1))
    by = np.unique(np.clip(by, 0, 1))
    for i in range(len(bx) - 1):
        a, b = bx[i], bx[i + 1]
        px = 0.5 * (b - a) * xs + 0.5 * (a + b)
        wx = 0.5 * (b - a) * ws
        for j in range(len(by) - 1):
            c, d = by[j], by[j + 1]
            py = 0.5 * (d - c) * xs + 0.5 * (c + d)
            wy = 0.5 * (d - c) * ws
            for u in range(order):
                for v in range(order):
                    tot += wx[u] * wy[v] * fun(np.array([px[u], py[v]]))
    return tot


# --------------------------------------------------------------------------
# A1: Philox4x32-10 -- published known-answer vectors (Salmon et al., SC'11)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key,expect", [
    ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
])
def test_philox_known_answers(oracle_mod, ctr, key, expect):
    assert list(oracle_mod.philox4x32_10(ctr, key)) == expect


def test_call_words_layout(oracle_mod):
    """Word w of a call = lane w%4 of block w/4 for counter (call, block,
    stream field, request) under key (seed lo, seed hi)."""
    pr = P.collider().replace(seed=0x1234567890ABCDEF, request_id=77)
    o = oracle_mod.Oracle(pr)
    o.allocate(1000)
    for call in (0, 1, 513, 959):
        r = o.eval_call(0, 5, call, with_bins=False)
        for w in range(pr.d):
            blk = oracle_mod.philox4x32_10([call, w // 4, 5, 77], [0x90ABCDEF, 0x12345678])
            assert r["words"][w] == blk[w % 4]
    r = o.eval_call(1, 0x80000000 | 3, 17, with_bins=False)
    for w in range(pr.d + 2):
        blk = oracle_mod.philox4x32_10([17, w // 4, 0x80000003, 77], [0x90ABCDEF, 0x12345678])
        assert r["words"][w] == blk[w % 4]


# --------------------------------------------------------------------------
# A3: forward grid map x = G^{-1}(r) on uniform and adapted grids (§3.2)
# --------------------------------------------------------------------------
def test_forward_map_uniform_grid_is_identity(oracle_mod):
    pr = P.single_gauss()
    o = oracle_mod.Oracle(pr)
    o.allocate(100)
    for call in range(100):
        r = o.eval_call(0, 0, call)
        u = (r["words"][: pr.d].astype(np.float64) + 0.5) / 2.0 ** 32
        np.testing.assert_allclose(r["x"], u, rtol=0, atol=2e-16)
        np.testing.assert_array_equal(r["jf"], np.floor(u * pr.n_bins).astype(int))


def test_forward_map_adapted_grid_inverse_cdf(oracle_mod):
    """On an adapted grid the point sits in bin j at fraction frac = u n - j,
    i.e. G(x) = r: the piecewise-linear CDF of the grid returns u."""
    pr = P.single_gauss()
    o = oracle_mod.Oracle(pr)
    adapt(o, pr, 3)
    e = o.get_state()["edges"][0]
    o.allocate(200)
    for call in range(200):
        r = o.eval_call(0, 9, call)
        u = (r["words"][: pr.d].astype(np.float64) + 0.5) / 2.0 ** 32
        for k in range(pr.d):
            j = r["jf"][k]
            assert e[k, j] <= r["x"][k] <= e[k, j + 1]
            cdf = (j + (r["x"][k] - e[k, j]) / (e[k, j + 1] - e[k, j])) / pr.n_bins
            assert abs(cdf - u[k]) < 1e-12


# --------------------------------------------------------------------------
# A4: channel maps -- round trip and Jacobian by finite differences (§3.4)
# --------------------------------------------------------------------------
def test_channel_maps_round_trip_and_jacobian(oracle_mod):
    pr = P.collider()
    o = oracle_mod.Oracle(pr)
    rng = np.random.default_rng(5)
    for c in range(0, pr.n_channels, 7):
        for _ in range(5):
            x = rng.uniform(0.05, 0.95, pr.d)
            p, jac = o.channel_forward(c, x)
            x2, jac2 = o.channel_inverse(c, p)
            # conditioning: dx/dp <= 1/(A Γ) ~ 3.2e3 at Γ = 1e-4, so a few ulp
            # of p become ~1e-12 in x
            np.testing.assert_allclose(x2, x, rtol=0, atol=3e-12)
            assert abs(jac2 / jac - 1) < 1e-10
            # 1/phi' = prod over mapped coordinates of dx/dp (finite differences)
            expect = 1.0
            for s in range(pr.channels.n_mapped[c]):
                k = pr.channels.coord[c, s]
                h = 1e-6 * max(x[k], 1e-3)
                xp, xm = x.copy(), x.copy()
                xp[k] += h
                xm[k] -= h
                dp = (o.channel_forward(c, xp)[0][k] - o.channel_forward(c, xm)[0][k]) / (2 * h)
                expect /= dp
            assert abs(jac / expect - 1) < 1e-6


# --------------------------------------------------------------------------
# A5: integrand normalisation, ∫ f = Σ w_k (quadrature at d = 2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pow_second", [False, True])
def test_integrand_normalised(oracle_mod, pow_second):
    pr = two_channel_problem(pow_second=pow_second)
    o = oracle_mod.Oracle(pr)
    bx = breakpoints_bw(0.37, 3e-3)
    by = (np.concatenate([np.linspace(0, 1, 61) ** 5, 0.55 ** np.arange(1, 180)])
          if pow_second else breakpoints_bw(0.61, 6e-3))
    tot = gl_integrate_2d(o.f, bx, by)
    assert abs(tot - 1.0) < 2e-7


def test_single_gauss_normalisation_closed_form(oracle_mod):
    """Config-1 integrand normalised on the real line: ∫_[0,1]^4 f = erf(...)^4.
    The 4-D integral factorises; check one axis by quadrature of f along a
    line through the centre and the others by the product rule."""
    pr = P.single_gauss()
    o = oracle_mod.Oracle(pr)
    xs, ws = leggauss(64)
    xs, ws = 0.5 * xs + 0.5, 0.5 * ws
    c = np.full(pr.d, 0.5)
    f0 = o.f(c)
    line = sum(w * o.f(np.array([x, 0.5, 0.5, 0.5])) for x, w in zip(xs, ws)) / f0
    expect_line = math.erf(0.5 / (0.1 * math.sqrt(2))) / (1.0 / (0.1 * math.sqrt(2 * math.pi)))
    assert abs(line - expect_line) < 1e-12
    assert abs(f0 - (0.1 * math.sqrt(2 * math.pi)) ** -4) < 1e-9


# --------------------------------------------------------------------------
# A6: densities are normalised: each g_c over x, and g(p) over p (Eqs. 26, 30)
# --------------------------------------------------------------------------
def test_grid_densities_normalised(oracle_mod):
    pr = two_channel_problem()
    o = oracle_mod.Oracle(pr)
    adapt(o, pr, 3)
    e = o.get_state()["edges"]
    for c in range(pr.n_channels):
        tot = 0.0
        for i in range(pr.n_bins):
            for j in range(pr.n_bins):
                mid = np.array([(e[c, 0, i] + e[c, 0, i + 1]) / 2, (e[c, 1, j] + e[c, 1, j + 1]) / 2])
                vol = (e[c, 0, i + 1] - e[c, 0, i]) * (e[c, 1, j + 1] - e[c, 1, j])
                tot += o.grid_density(c, mid) * vol
        assert abs(tot - 1.0) < 1e-12


@pytest.mark.parametrize("pow_second", [False, True])
def test_multichannel_density_normalised(oracle_mod, pow_second):
    pr = two_channel_problem(pow_second=pow_second)
    o = oracle_mod.Oracle(pr)
    adapt(o, pr, 3)
    stt = o.get_state()
    assert np.all(np.abs(stt["alpha"] - 0.5) > 1e-3)  # α really adapted
    e = stt["edges"]
    # breakpoints: images in p of every channel's x-edges, plus resolution
    bx = [breakpoints_bw(0.37, 3e-3, n=100)]
    # the power-law Jacobian 0.2 p^-0.8 is singular at 0: geometric cells
    by = [np.concatenate([np.linspace(0, 1, 61) ** 5, 0.55 ** np.arange(1, 180)])
          if pow_second else breakpoints_bw(0.61, 6e-3, n=100)]
    for c in range(2):
        for k, acc in ((0, bx), (1, by)):
            pts = []
            for xe in e[c, k]:
                x = np.full(2, 0.5)
                x[k] = xe
                pts.append(o.channel_forward(c, x)[0][k])
            acc.append(np.array(pts))
    tot = gl_integrate_2d(o.g, np.concatenate(bx), np.concatenate(by), order=6)
    assert abs(tot - 1.0) < 1e-6


# --------------------------------------------------------------------------
# Closed-form special cases of the whole pass (w ≡ 1)
# --------------------------------------------------------------------------
def test_constant_integrand_exact(oracle_mod):
    pr = P.special_case("const", d=3)
    o = oracle_mod.Oracle(pr)
    r = o.sample_pass(5000, 0)
    # w = 1 up to the rounding of 1/(n Δx) on the uniform grid
    assert abs(r.integral - 1.0) < 1e-14 and r.variance < 1e-28
    assert abs(r.w_max - 1.0) < 1e-14 and abs(r.efficiency - 1.0) < 1e-14
    assert r.n_calls == 5000


@pytest.mark.parametrize("kind", ["bw", "pow"])
def test_mapped_peak_gives_unit_weight(oracle_mod, kind):
    pr = P.special_case(kind, d=2)
    o = oracle_mod.Oracle(pr)
    r = o.sample_pass(5000, 0)
    assert abs(r.integral - 1.0) < 1e-13
    assert r.variance < 1e-28
    assert abs(r.w_max - 1.0) < 1e-13


def test_identical_channels_equal_single_channel(oracle_mod):
    """K identical channels: every weight and the integral equal those of the
    single-channel run on the same random words, whatever α is."""
    base = two_channel_problem()
    one = base.replace(channels=P.MapSet(*(np.array(getattr(base.channels, f))[:1] for f in
                                           ("n_mapped", "coord", "kind", "a", "b"))))
    K = 4
    many = base.replace(channels=P.MapSet(*(np.repeat(np.array(getattr(base.channels, f))[:1], K, 0)
                                            for f in ("n_mapped", "coord", "kind", "a", "b"))))
    o1, oK = oracle_mod.Oracle(one), oracle_mod.Oracle(many)
    N = 4000
    r1 = o1.sample_pass(N, 0)
    rK = oK.sample_pass(N, 0)
    assert abs(rK.integral / r1.integral - 1) < 1e-13
    o1.allocate(N)
    for alpha in (np.full(K, 0.25), np.array([0.1, 0.2, 0.3, 0.4])):
        oK.set_state(alpha=alpha, have_pass=True)
        oK.allocate(N)
        for call in (0, 999, 1000, 2500, 3999):
            a, b = o1.eval_call(0, 3, call), oK.eval_call(0, 3, call)
            if b["channel"] >= 0:
                assert abs(a["w"] / b["w"] - 1) < 1e-13


# --------------------------------------------------------------------------
# A7/A8: accumulation and estimators, brute force on a tiny pass
# --------------------------------------------------------------------------
def test_pass_sums_brute_force(oracle_mod):
    pr = two_channel_problem(n_bins=5)
    o = oracle_mod.Oracle(pr)
    adapt(o, pr, 2, calls=400)
    stt = o.get_state()
    alpha, shift = stt["alpha"], stt["shift"]
    N, it = 300, 7
    Nt = o.allocate(N)
    calls = [o.eval_call(0, it, i, with_bins=False) for i in range(Nt)]
    r = o.sample_pass(N, it)
    ps = o.get_pass()
    D = np.zeros((2, pr.d, pr.n_bins))
    I = 0.0
    V = 0.0
    wmax = 0.0
    for c in range(2):
        w = np.array([x["w"] for x in calls if x["channel"] == c])
        assert len(w) == ps["Nc"][c]
        assert abs(np.mean(w) - ps["Ic"][c]) <= 1e-13 * abs(np.mean(w))
        assert abs(np.var(w, ddof=1) - ps["Vc"][c]) <= 1e-12 * np.mean(w ** 2)
        I += alpha[c] * np.mean(w)
        V += alpha[c] ** 2 * np.var(w, ddof=1) / len(w)
        wmax = max(wmax, w.max())
    for x in calls:
        for k in range(pr.d):
            D[x["channel"], k, x["jf"][k]] += x["w"] ** 2
    np.testing.assert_allclose(ps["D"], D, rtol=1e-13, atol=0)
    assert abs(r.integral - I) <= 1e-13 * I
    assert abs(r.variance - V) <= 1e-12 * V
    assert r.w_max == wmax
    assert abs(r.efficiency - I / wmax) < 1e-15
    assert np.all(shift != 0)  # the shifted sums were really exercised


def test_bin_dvalues_expectation_by_quadrature(oracle_mod):
    """E[D_{k,j}] = N ∫_{x_k in bin j} f²/g dx (Eq. 15, ρ = 1): single identity
    channel, uniform grid (g = 1), Gaussian integrand; mean over seeds."""
    pr = P.single_gauss().replace(d=2, n_bins=4, gauss_sigma=0.3)
    N = 4000
    acc = []
    for s in range(30):
        o = oracle_mod.Oracle(pr.replace(seed=500 + s))
        o.sample_pass(N, 0)
        acc.append(o.get_pass()["D"][0, 0])
    acc = np.array(acc)
    from scipy.special import erf
    sg = 0.3
    z = 1.0 / (sg * math.sqrt(2 * math.pi))
    # ∫ G² over an interval: G² = z² exp(-(x-.5)²/σ²) -> z² σ √π/2 [erf]
    def int_g2(a, b):
        return z * z * sg * math.sqrt(math.pi) / 2 * (erf((b - 0.5) / sg) - erf((a - 0.5) / sg))
    other = int_g2(0.0, 1.0)
    edges = np.linspace(0, 1, 5)
    expect = np.array([N * int_g2(edges[j], edges[j + 1]) * other for j in range(4)])
    sem = acc.std(axis=0, ddof=1) / math.sqrt(len(acc))
    assert np.all(np.abs(acc.mean(axis=0) - expect) < 4 * sem)


# --------------------------------------------------------------------------
# Unbiasedness: estimator mean over 100 seeds within 3σ of the exact value
# --------------------------------------------------------------------------
def _seed_study(oracle_mod, make, exact, iters, calls, seeds=100):
    per_iter = [[] for _ in range(iters)]
    for s in range(seeds):
        pr = make(s)
        o = oracle_mod.Oracle(pr)
        for it in range(iters):
            r = o.sample_pass(calls, it, n_threads=1)
            per_iter[it].append(r.integral)
            o.refine_grids()
            if pr.adapt_alpha:
                o.update_alpha()
    for it in range(iters):
        a = np.array(per_iter[it])
        z = (a.mean() - exact) / (a.std(ddof=1) / math.sqrt(len(a)))
        assert abs(z) < 3.0, (it, a.mean(), exact, z)


def test_unbiased_single_gauss(oracle_mod):
    exact = math.erf(0.5 / (0.1 * math.sqrt(2))) ** 4
    _seed_study(oracle_mod, lambda s: P.single_gauss(seed=100 + s), exact, 5, 10_000)


def test_unbiased_bw_gauss(oracle_mod):
    _seed_study(oracle_mod, lambda s: P.bw_gauss(rng_seed=200 + s), 1.0, 3, 20_000)


def test_unbiased_collider_reduced(oracle_mod):
    _seed_study(oracle_mod, lambda s: P.collider(rng_seed=300 + s), 1.0, 1, 2_000, seeds=60)


# --------------------------------------------------------------------------
# A9: rebinning (Eqs. 14, 15) -- mpmath root finding + invariants
# --------------------------------------------------------------------------
def _mp_refine(D, edges, alpha):
    import mpmath as mp
    mp.mp.dps = 40
    n = len(D)
    om = [mp.sqrt(mp.mpf(v)) for v in D]
    S = mp.fsum(om)
    m = []
    for o_ in om:
        r = o_ / S
        m.append(mp.mpf(0) if r == 0 else ((r - 1) / mp.log(r)) ** alpha)
    M = mp.fsum(m)
    e = [mp.mpf(v) for v in edges]

    def cdf(x):  # cumulative of m, linear inside each old bin
        tot = mp.mpf(0)
        for j in range(n):
            if x >= e[j + 1]:
                tot += m[j]
            elif x > e[j]:
                tot += m[j] * (x - e[j]) / (e[j + 1] - e[j])
        return tot / M

    out = [mp.mpf(0)]
    for i in range(1, n):
        out.append(mp.findroot(lambda x: cdf(x) - mp.mpf(i) / n, (e[0], e[-1]), solver="bisect",
                               tol=mp.mpf(10) ** -35, maxsteps=400))
    out.append(mp.mpf(1))
    return np.array([float(v) for v in out])


@pytest.mark.parametrize("alpha", [1.0, 1.5])
@pytest.mark.parametrize("D,edges", [
    ([1.0, 4.0, 9.0, 16.0], [0.0, 0.25, 0.5, 0.75, 1.0]),
    ([0.3, 0.0, 2.5, 0.7], [0.0, 0.1, 0.45, 0.8, 1.0]),
    ([5.0, 1e-6, 1e-6, 5.0], [0.0, 0.4, 0.5, 0.6, 1.0]),
])
def test_refine_worked_examples(oracle_mod, alpha, D, edges):
    got = oracle_mod.refine_row(D, edges, alpha_grid=alpha)
    exp = _mp_refine(D, edges, alpha)
    np.testing.assert_allclose(got, exp, rtol=0, atol=1e-14)


def test_refine_direction_and_invariants(oracle_mod):
    rng = np.random.default_rng(3)
    n = 50
    for _ in range(50):
        e = np.sort(np.concatenate([[0, 1], rng.uniform(0, 1, n - 1)]))
        D = rng.exponential(1.0, n) * (rng.uniform(size=n) > 0.2)
        ne = oracle_mod.refine_row(D, e, alpha_grid=1.5)
        assert ne[0] == 0.0 and ne[-1] == 1.0
        assert np.all(np.diff(ne) > 0)
    # uniform D on a uniform grid: unchanged to an ulp
    e = np.linspace(0, 1, n + 1)
    ne = oracle_mod.refine_row(np.full(n, 2.0), e, alpha_grid=1.5)
    np.testing.assert_allclose(ne, e, rtol=0, atol=2.3e-16)
    # all-zero row: unchanged
    assert np.array_equal(oracle_mod.refine_row(np.zeros(n), e), e)
    # the bin with the largest weight gets narrower, the smallest wider
    D = np.ones(n)
    D[10] = 100.0
    D[30] = 1e-4
    ne = oracle_mod.refine_row(D, e, alpha_grid=1.5)
    w = np.diff(ne)
    ow = np.diff(e)
    # the region of the heavy bin gets more edges: edges crowd around 0.2-0.22
    assert np.sum((ne > 0.2) & (ne < 0.22)) > 1
    assert w.min() < ow.min()


def test_refine_smoothing(oracle_mod):
    """Smoothing replaces D by its 3-point average before ω (reading): the
    smoothed refine equals the plain refine of the averaged row."""
    D = np.array([1.0, 8.0, 2.0, 0.5, 4.0])
    e = np.linspace(0, 1, 6)
    avg = np.array([(D[0] + D[1]) / 2, (D[0] + D[1] + D[2]) / 3, (D[1] + D[2] + D[3]) / 3,
                    (D[2] + D[3] + D[4]) / 3, (D[3] + D[4]) / 2])
    a = oracle_mod.refine_row(D, e, smooth=1)
    b = oracle_mod.refine_row(avg, e, smooth=0)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# A2/A10: allocation and channel-weight update (Eq. 25)
# --------------------------------------------------------------------------
def test_allocation(oracle_mod):
    nc, pc = oracle_mod.allocate([0.5, 0.3, 0.2, 0.0], 1000)
    assert list(nc) == [500, 300, 200, 0] and list(pc) == [0, 500, 800, 1000, 1000]
    nc, _ = oracle_mod.allocate([0.999, 0.001], 1000, n_min=10)
    assert list(nc) == [999, 10]
    nc, _ = oracle_mod.allocate([1 / 3] * 3, 100)
    assert list(nc) == [33, 33, 33]
    nc, _ = oracle_mod.allocate([0.6666, 0.3334], 1000)  # floor, not rounding (R6)
    assert list(nc) == [666, 333]


def test_alpha_update_properties(oracle_mod):
    a = np.array([0.5, 0.3, 0.2])
    N = np.array([100, 100, 100])
    # equal ω: fixed point
    np.testing.assert_allclose(oracle_mod.alpha_update(a, [2.0, 2.0, 2.0], [1, 1, 1], N), a,
                               rtol=1e-15)
    # ratio rule α'_1/α'_2 = (α_1/α_2)(ω_1/ω_2)^β for β = 0.5 and β = 1
    for beta in (0.5, 1.0):
        out = oracle_mod.alpha_update(a, [4.0, 1.0, 9.0], [1, 1, 1], N, beta=beta)
        assert abs(out.sum() - 1) < 1e-15
        assert abs(out[0] / out[1] - (0.5 / 0.3) * 4.0 ** beta) < 1e-12
        assert abs(out[2] / out[1] - (0.2 / 0.3) * 9.0 ** beta) < 1e-12
    # a channel whose calls all gave w = 0 is switched off
    out = oracle_mod.alpha_update(a, [4.0, 1.0, 0.0], [1, 1, 0.0], N)
    assert out[2] == 0.0 and abs(out.sum() - 1) < 1e-15
    # a channel without variance but with a non-zero mean keeps its share
    out = oracle_mod.alpha_update(a, [4.0, 1.0, 0.0], [1, 1, 2.0], N)
    assert abs(out[2] - 0.2) < 1e-15 and abs(out.sum() - 1) < 1e-15
    # switched-off channels stay off
    out = oracle_mod.alpha_update([0.5, 0.5, 0.0], [1.0, 4.0, 3.0], [1, 1, 1], [10, 10, 0])
    assert out[2] == 0.0


def test_alpha_adaptation_moves_towards_larger_variance(oracle_mod):
    pr = P.bw_gauss()
    o = oracle_mod.Oracle(pr)
    o.sample_pass(20_000, 0)
    ps = o.get_pass()
    o.update_alpha()
    a = o.get_state()["alpha"]
    order_v = np.argsort(ps["Vc"])
    order_a = np.argsort(a)
    assert np.array_equal(order_v, order_a)


# --------------------------------------------------------------------------
# A11: combination of iterations (inverse-variance weights)
# --------------------------------------------------------------------------
def test_combination_inverse_variance(oracle_mod):
    pr = P.single_gauss()
    o = oracle_mod.Oracle(pr)
    Is, Vs = [], []
    r = None
    for it in range(5):
        comb = it >= 2
        r = o.sample_pass(5000, it, combine=comb)
        if comb:
            Is.append(r.integral)
            Vs.append(r.variance)
        o.refine_grids()
    Is, Vs = np.array(Is), np.array(Vs)
    w = 1 / Vs
    Ibar = np.sum(w * Is) / np.sum(w)
    assert abs(r.combined - Ibar) < 1e-14
    assert abs(r.combined_sigma - np.sqrt(1 / np.sum(w))) < 1e-16
    assert abs(r.chi2_dof - np.sum((Is - Ibar) ** 2 * w) / (len(Is) - 1)) < 1e-12


# --------------------------------------------------------------------------
# A12: unweighted generation
# --------------------------------------------------------------------------
def test_generation_channel_choice_frequencies(oracle_mod):
    pr = P.bw_gauss()
    o = oracle_mod.Oracle(pr)
    o.sample_pass(20_000, 0)
    o.update_alpha()
    a = o.get_state()["alpha"]
    counts = np.zeros(pr.n_channels)
    for i in range(6000):
        counts[o.eval_call(1, 0x80000000, i, with_bins=False)["channel"]] += 1
    chi2 = np.sum((counts - 6000 * a) ** 2 / (6000 * a))
    assert st.chi2.sf(chi2, pr.n_channels - 1) > 1e-3


def test_generation_brute_force_order_and_batches(oracle_mod):
    pr = two_channel_problem(n_bins=6).replace(gen_batch=256)
    o = oracle_mod.Oracle(pr)
    adapt(o, pr, 2, calls=2000)
    # lower w_max so that overweights happen and the between-batch raise matters
    stt = o.get_state()
    wm0 = 0.3 * stt["w_max"]
    o.set_state(w_max=wm0, have_pass=True)
    res = o.generate(300, gen_id=5)
    wm = wm0
    got_p, got_w, used, over, b = [], [], 0, 0, 0
    while len(got_w) < 300:
        field = 0x80000000 | (5 << 16) | b
        bmax = 0.0
        for i in range(256):
            r = o.eval_call(1, field, i, with_bins=False)
            u = (float(r["words"][pr.d + 1]) + 0.5) / 2 ** 32
            bmax = max(bmax, r["w"])
            if len(got_w) < 300:
                used += 1
                if u * wm < r["w"]:
                    got_p.append(r["p"].astype(np.float32))
                    got_w.append(r["w"])
                    over += r["w"] > wm
        wm = max(wm, bmax)
        b += 1
    assert res["n_written"] == 300 and res["n_calls_used"] == used
    assert res["n_overweight"] == over and over > 0 and res["n_batches"] == b
    np.testing.assert_array_equal(res["w"], np.array(got_w))
    np.testing.assert_array_equal(res["p"], np.array(got_p))
    assert abs(o.get_state()["w_max"] - wm) == 0


def test_generation_marginals_match_integrand(oracle_mod):
    """Accepted events follow f: KS test of both 1-D marginals against the
    closed-form CDFs of the normalised integrand (no overweights allowed)."""
    pr = two_channel_problem(n_bins=20).replace(gen_batch=1 << 14)
    o = oracle_mod.Oracle(pr)
    adapt(o, pr, 4, calls=20_000)
    o.set_state(w_max=2.0 * o.get_state()["w_max"], have_pass=True)
    res = o.generate(3000, gen_id=1)
    assert res["n_overweight"] == 0
    p = res["p"].astype(np.float64)

    def cdf0(x):
        return 0.6 * bw_cdf(x, 0.37, 3e-3) + 0.4 * tgauss_cdf(x)

    def cdf1(x):
        return 0.6 * tgauss_cdf(x) + 0.4 * bw_cdf(x, 0.61, 6e-3)

    assert st.kstest(p[:, 0], cdf0).pvalue > 1e-3
    assert st.kstest(p[:, 1], cdf1).pvalue > 1e-3
    # acceptance rate = E[min(w, w_max)] / w_max = I / w_max without overweights
    rate = res["n_written"] / res["n_calls_used"]
    expect = 1.0 / o.get_state()["w_max"]
    assert abs(rate - expect) < 4 * math.sqrt(expect * (1 - expect) / res["n_calls_used"])


def test_generation_channel_choice_is_inverse_cdf(oracle_mod):
    """Convention check (no statistical signature): the channel of a
    generation call is the inverse CDF of the cumulative α at the uniform
    u = (X_d + 1/2) 2^-32 of word d."""
    pr = P.bw_gauss()
    o = oracle_mod.Oracle(pr)
    o.set_state(alpha=np.array([0.05, 0.1, 0.15, 0.2, 0.22, 0.28]), have_pass=True)
    A = np.cumsum(o.get_state()["alpha"])
    for i in range(3000):
        r = o.eval_call(1, 0x80000007, i, with_bins=False)
        u = (float(r["words"][pr.d]) + 0.5) * 2.0 ** -32
        c = r["channel"]
        assert u * A[-1] < A[c] and (c == 0 or u * A[-1] >= A[c - 1])


@pytest.mark.parametrize("factory,calls", [(P.bw_gauss, 60_000), (P.collider, 6_000)])
def test_thread_split_is_exact(oracle_mod, factory, calls):
    """The oracle's multi-threaded pass (contiguous call chunks, ordered merge
    of compensated partial sums) equals its single-threaded pass."""
    pr = factory()
    a, b = oracle_mod.Oracle(pr), oracle_mod.Oracle(pr)
    for it in range(2):
        ra = a.sample_pass(calls, it, n_threads=1)
        rb = b.sample_pass(calls, it, n_threads=7)
        assert ra.n_calls == rb.n_calls and ra.w_max == rb.w_max
        assert abs(ra.integral - rb.integral) <= 1e-15 * abs(ra.integral)
        assert abs(ra.variance - rb.variance) <= 1e-13 * ra.variance
        Da, Db = a.get_pass()["D"], b.get_pass()["D"]
        assert np.abs(Da - Db).max() <= 1e-14 * Da.max()
        for o in (a, b):
            o.refine_grids()
            o.update_alpha()


def test_bin_rule_at_edges(oracle_mod):
    """R11: x in bin j iff ξ_j <= x < ξ_{j+1}; a point on an interior edge
    belongs to the upper bin, x = 1 to the last bin (density 1/(n Δx_j),
    Eq. 12)."""
    pr = P.special_case("const", d=1, n_bins=5)
    o = oracle_mod.Oracle(pr)
    e = np.array([0.0, 0.1, 0.25, 0.6, 0.7, 1.0])
    o.set_state(e.reshape(1, 1, 6), np.ones(1), np.zeros(1), 0.0, have_pass=True)
    dens = 1.0 / (5 * np.diff(e))
    for j in range(1, 5):
        assert o.grid_density(0, [e[j]]) == dens[j]
        assert o.grid_density(0, [np.nextafter(e[j], 0.0)]) == dens[j - 1]
    assert o.grid_density(0, [1.0]) == dens[4]
    assert o.grid_density(0, [0.0]) == dens[0]


def test_power_map_clamp_at_zero(oracle_mod):
    """R15: where x^5 underflows (or x = 0) the power map gives p = the
    smallest normal double, not 0, so that the integrand factor and the
    other channels' inverse maps stay finite; above that p = x^5."""
    o = oracle_mod.Oracle(P.special_case("pow", d=2))
    tiny = np.finfo(np.float64).tiny
    p, _ = o.channel_forward(0, [0.0, 0.5])
    assert p[0] == tiny and p[1] == 0.5
    p, jac = o.channel_forward(0, [1e-70, 0.5])  # (1e-70)^5 underflows
    assert p[0] == tiny and np.isfinite(jac) and jac > 0.0
    assert np.isfinite(o.f(p)) and np.isfinite(o.g(p))
    p, _ = o.channel_forward(0, [0.5, 0.5])
    assert p[0] == 0.5 ** 5


def test_smoothing_is_the_three_point_average(oracle_mod):
    """R3: smooth = 1 rebins from (D_1 + D_2)/2, (D_{j-1} + D_j + D_{j+1})/3,
    (D_{n-1} + D_n)/2 -- the same edges as rebinning the averaged row."""
    rng = np.random.default_rng(4)
    n = 12
    e = np.sort(np.concatenate([[0, 1], rng.uniform(0, 1, n - 1)]))
    D = rng.exponential(1.0, n)
    avg = np.empty(n)
    avg[0] = (D[0] + D[1]) / 2
    avg[-1] = (D[-2] + D[-1]) / 2
    avg[1:-1] = (D[:-2] + D[1:-1] + D[2:]) / 3
    got = oracle_mod.refine_row(D, e, alpha_grid=1.5, smooth=1)
    ref = oracle_mod.refine_row(avg, e, alpha_grid=1.5, smooth=0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)
    assert np.abs(got - oracle_mod.refine_row(D, e, alpha_grid=1.5, smooth=0)).max() > 1e-4

"""Pins of the oracle's pseudo-stratified mode (§3.3; readings R16, R17)
against facts fixed by the definition and by statistics (CPU only)."""
import math

import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P


@pytest.mark.parametrize("N,d", [(1, 1), (2, 1), (3, 1), (1000, 2), (999, 2), (10_000, 4), (156_250, 14),
                                 (10, 4), (2 ** 18, 3), (7, 2), (2 * 5 ** 6, 6), (2 * 5 ** 6 - 1, 6)])
def test_cells_per_axis_brute_force(oracle_mod, N, d):
    m = oracle_mod.strat_cells_per_axis(N, d)
    best = 1
    for cand in range(1, 2000):
        if 2 * cand ** d <= N:
            best = cand
    assert m == max(1, best)
    assert m == 1 or 2 * m ** d <= N


def test_cells_per_axis_cap(oracle_mod):
    assert oracle_mod.strat_cells_per_axis(2 ** 40, 1) == 2 ** 20


def test_allocation_whole_cells(oracle_mod):
    """N_c = s C with C = n_r^d and s = floor(N_c / C) >= 2 cells' worth."""
    pr = P.bw_gauss().replace(stratified=1)
    o = oracle_mod.Oracle(pr)
    N = 200_000
    raw = oracle_mod.allocate(np.full(pr.n_channels, 1.0 / pr.n_channels), N, pr.n_min)[0]
    total = o.allocate(N)
    ps = o.get_pass()
    expect = 0
    for nc in raw:
        m = oracle_mod.strat_cells_per_axis(nc, pr.d)
        C = m ** pr.d
        expect += (nc // C) * C
    assert total == expect and ps["Nc"].sum() == total


def test_one_cell_per_channel_is_importance_sampling(oracle_mod):
    """n_r = 1 (N_c < 2^(d+1)): r_k = u_k as in R10 and the variance of R17
    is the ordinary sample variance: the pass equals importance sampling."""
    pr = P.bw_gauss()  # d = 8, K = 6: N_c ~ 66 < 512
    a = oracle_mod.Oracle(pr).sample_pass(400, 3, n_threads=1)
    b = oracle_mod.Oracle(pr.replace(stratified=1)).sample_pass(400, 3, n_threads=2)
    assert a.n_calls == b.n_calls
    assert a.integral == b.integral
    assert abs(a.variance - b.variance) <= 1e-13 * a.variance
    assert a.w_max == b.w_max


def test_points_lie_in_their_cells(oracle_mod):
    """Identity channel on uniform grids: p = x = r, so call l of the channel
    lies in r cell floor(l / s) with base-n_r digits a_k."""
    pr = P.special_case("const", d=3, n_bins=7).replace(stratified=1)
    o = oracle_mod.Oracle(pr)
    N = o.allocate(5000)
    m = oracle_mod.strat_cells_per_axis(5000, 3)
    C = m ** 3
    s = 5000 // C
    assert N == s * C and s >= 2
    seen = np.zeros(C, np.int64)
    for call in range(N):
        ev = o.eval_call(0, 9, call, with_bins=False)
        cell = call // s
        digits = [(cell // m ** k) % m for k in range(3)]
        for k in range(3):
            assert digits[k] / m <= ev["p"][k] < (digits[k] + 1) / m
        seen[cell] += 1
        assert abs(ev["w"] - 1.0) < 1e-14
    assert (seen == s).all()


def test_constant_integrand_zero_variance(oracle_mod):
    pr = P.special_case("const", d=2, n_bins=4).replace(stratified=1)  # Δx = 1/4: densities exactly 1
    r = oracle_mod.Oracle(pr).sample_pass(10_000, 0, n_threads=3)
    assert r.integral == 1.0 and r.variance == 0.0


def test_stratified_unbiased_and_error_estimate_consistent(oracle_mod):
    """Over 80 seeds: the mean is within 3σ of the exact integral, and the
    pass's own σ estimate (R17) matches the spread of the estimates."""
    exact = math.erf(0.5 / (0.1 * math.sqrt(2))) ** 4
    est, sig = [], []
    for s in range(80):
        pr = P.single_gauss(seed=500 + s).replace(stratified=1)
        r = oracle_mod.Oracle(pr).sample_pass(20_000, 0, n_threads=1)
        est.append(r.integral)
        sig.append(math.sqrt(r.variance))
    est, sig = np.array(est), np.array(sig)
    z = (est.mean() - exact) / (est.std(ddof=1) / math.sqrt(len(est)))
    assert abs(z) < 3.0
    ratio = est.std(ddof=1) / np.sqrt(np.mean(sig ** 2))
    assert 0.75 < ratio < 1.3, ratio


def test_stratified_reduces_error_on_a_smooth_integrand(oracle_mod):
    """Same calls budget, uniform grids: stratification in r space lowers the
    error of a smooth integrand (averaged over seeds)."""
    imp, strat = [], []
    for s in range(20):
        pr = P.single_gauss(seed=700 + s)
        imp.append(oracle_mod.Oracle(pr).sample_pass(20_000, 0, n_threads=1).variance)
        strat.append(oracle_mod.Oracle(pr.replace(stratified=1)).sample_pass(20_000, 0, n_threads=1).variance)
    assert np.mean(strat) < 0.6 * np.mean(imp)


def test_thread_split_by_cells_is_exact(oracle_mod):
    pr = P.bw_gauss().replace(stratified=1)
    a = oracle_mod.Oracle(pr).sample_pass(100_000, 1, n_threads=1)
    b = oracle_mod.Oracle(pr).sample_pass(100_000, 1, n_threads=7)
    assert a.n_calls == b.n_calls
    assert abs(a.integral - b.integral) <= 1e-15 * abs(a.integral)
    assert abs(a.variance - b.variance) <= 1e-12 * a.variance

"""Pins of the oracle on integrands of both signs (§3.1; reading R19) against
facts fixed by the integrand (closed-form integral, quadrature of |f|) and
by brute force (CPU only)."""
import math

import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P


def _abs_f_table(o, n=8001):
    """Fine grid on [0, 1], f and the normalised CDF of |f| (Simpson)."""
    x = np.linspace(0.0, 1.0, n)
    f = np.array([o.f([t]) for t in x])
    a = np.abs(f)
    h = x[1] - x[0]
    # cumulative Simpson on pairs of intervals, trapezoid inside a pair
    cum = np.zeros(n)
    cum[1:] = np.cumsum(0.5 * h * (a[1:] + a[:-1]))
    simpson = h / 3.0 * (a[0] + a[-1] + 4.0 * a[1:-1:2].sum() + 2.0 * a[2:-1:2].sum())
    return x, f, cum / cum[-1], simpson


def test_signed_integral_unbiased_and_error_consistent(oracle_mod):
    """f = 1.3 BW(0.3) - 0.3 BW(0.7): the integral is 1.0 exactly; over 60
    seeds the mean is within 3σ and the passes' own σ match the spread."""
    est, sig = [], []
    for s in range(60):
        o = oracle_mod.Oracle(P.signed_pair(d=2, seed=300 + s))
        r = o.sample_pass(20_000, 0, n_threads=1)
        est.append(r.integral)
        sig.append(math.sqrt(r.variance))
    est, sig = np.array(est), np.array(sig)
    z = (est.mean() - 1.0) / (est.std(ddof=1) / math.sqrt(len(est)))
    assert abs(z) < 3.0, z
    ratio = est.std(ddof=1) / np.sqrt(np.mean(sig ** 2))
    assert 0.75 < ratio < 1.3, ratio


def test_signed_adapted_run_converges_to_the_signed_sum(oracle_mod):
    pr = P.signed_bw_gauss()
    o = oracle_mod.Oracle(pr)
    for it in range(6):
        r = o.sample_pass(200_000, it, combine=it >= 2, n_threads=4)
        o.refine_grids()
        o.update_alpha()
    exact = float(pr.peak_weight.sum())
    assert abs(r.combined - exact) < 4.0 * r.combined_sigma, (r.combined, exact, r.combined_sigma)


def test_w_max_is_the_largest_abs_weight(oracle_mod):
    """Brute force over every call of a pass: w_max = max |w|, and here the
    largest |w| belongs to a negative weight (max w is far below it)."""
    o = oracle_mod.Oracle(P.signed_pair(weights=(-1.3, 0.3), d=2))
    r = o.sample_pass(3000, 4, n_threads=2)
    w = np.array([o.eval_call(0, 4, i, with_bins=False)["w"] for i in range(r.n_calls)])
    assert r.w_max == np.abs(w).max()
    assert w.max() < 0.5 * r.w_max and w.min() < 0.0


def test_signed_events_follow_abs_f_and_keep_the_sign(oracle_mod):
    """Accepted events are distributed as |f| (KS against the quadrature CDF),
    carry the sign of f at their point, and the mean sign is ∫f / ∫|f|."""
    pr = P.signed_pair(weights=(1.3, -0.3), d=1).replace(gen_batch=1 << 14)
    o = oracle_mod.Oracle(pr)
    for it in range(4):
        o.sample_pass(20_000, it, n_threads=2)
        o.refine_grids()
        o.update_alpha()
    o.set_state(w_max=2.0 * o.get_state()["w_max"], have_pass=True)
    n = 4000
    res = o.generate(n, gen_id=3)
    assert res["n_written"] == n and res["n_overweight"] == 0
    p = res["p"][:, 0].astype(np.float64)
    w = res["w"]
    x, f, cdf, abs_int = _abs_f_table(o)
    fp = np.array([o.f([t]) for t in p])
    assert np.all(np.sign(w) == np.sign(fp))
    # KS distance of the events against the CDF of |f|
    ps = np.sort(p)
    F = np.interp(ps, x, cdf)
    ecdf_hi = np.arange(1, n + 1) / n
    ks = max(np.abs(ecdf_hi - F).max(), np.abs(ecdf_hi - 1.0 / n - F).max())
    assert ks < 1.63 / math.sqrt(n), ks  # 1 % level
    # mean sign
    m = float(np.mean(np.sign(w)))
    expect = 1.0 / abs_int  # ∫f = 1
    assert abs(m - expect) < 4.0 * math.sqrt((1.0 - expect ** 2) / n), (m, expect)
    assert (w < 0).sum() > 0.05 * n


def test_generation_raises_w_max_to_the_largest_abs_weight(oracle_mod):
    """With w_max set too low, generation raises it between batches to the
    largest |w| seen: it ends at or above every event's |w|, also when the
    largest ones are negative."""
    pr = P.signed_pair(weights=(-1.3, 0.3), d=2).replace(gen_batch=512)
    o = oracle_mod.Oracle(pr)
    for it in range(2):
        o.sample_pass(5000, it, n_threads=2)
        o.refine_grids()
    wm0 = 0.05 * o.get_state()["w_max"]
    o.set_state(w_max=wm0, have_pass=True)
    res = o.generate(2000, gen_id=2)
    wm = o.get_state()["w_max"]
    assert res["n_overweight"] > 0 and res["n_batches"] >= 2
    assert wm >= np.abs(res["w"]).max()
    assert np.abs(res["w"][res["w"] < 0]).max() > res["w"].max()

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (stated per test):
  * integer / index work -- random words, channel choices, forward and
    inverse bin indices, call counts, event order: bit-exact;
  * FP64 path: weights, sums, integral, variance, refined edges, α within
    1e-12 relative (variance relative to the second moment, because the
    variance of well-adapted passes is a difference of nearly equal sums);
  * FP32-eval path: pass integral within 1e-6 relative and 0.05 σ of the
    oracle's estimate on the same state; per-call weights within a few
    float ulps except where an FP32 coordinate falls in a different bin.
"""
import math
import os

import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1811_09711_gb300 import vamp
    vamp.load()
    return vamp


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) if a.size else 0.0


def run_schedule(V, O, pr, iters, calls, prec=0, check=True, tol=1e-12):
    g = V.Vamp(pr, precision=prec)
    o = O.Oracle(pr)
    out = []
    for it in range(iters):
        comb = it >= pr.combine_from
        s_prev = o.get_state()["shift"]  # shift s_c the pass's sums are taken about
        rg = g.sample_pass(calls, it)
        ro = o.sample_pass(calls, it, combine=comb, n_threads=NTHREADS)
        out.append((rg, ro))
        if check:
            assert rg.n_calls == ro.n_calls
            assert rel(rg.integral, ro.integral) < tol, (it, rg.integral, ro.integral)
            m2 = ro.variance + ro.integral ** 2 / max(ro.n_calls, 1)
            assert abs(rg.variance - ro.variance) <= tol * max(m2, 1e-300), (it, rg.variance, ro.variance)
            assert rel(rg.w_max, ro.w_max) < tol
            if comb:
                assert rel(rg.combined, ro.combined) < tol
            pg, po = g.get_pass(), o.get_pass()
            assert np.array_equal(pg["Nc"], po["Nc"])
            np.testing.assert_allclose(pg["D"], po["D"], rtol=tol, atol=tol * po["D"].max())
            # α_c ∝ V_c^β, and V_c comes from sums shifted by s_c: the
            # difference of the shifted moments loses a factor
            # (V_c + (I_c - s_c)^2) / V_c to cancellation, which α inherits
            live = (po["Nc"] > 1) & (po["Vc"] > 0)
            m2s = po["Vc"][live] + (po["Ic"][live] - s_prev[live]) ** 2
            cond = float(np.max(m2s / po["Vc"][live])) if live.any() else 1.0
        if pr.adapt_grid:
            g.refine_grids()
            o.refine_grids()
        if pr.adapt_alpha:
            g.update_alpha()
            o.update_alpha()
        if check:
            sg, so = g.get_state(), o.get_state()
            np.testing.assert_allclose(sg["edges"], so["edges"], rtol=0, atol=tol)
            assert rel(sg["alpha"], so["alpha"]) < tol * max(1.0, cond), (it, cond)
    return g, o, out


# --------------------------------------------------------------------------
# bit-exact integer work: channels, forward bins, every channel's bin lookup
# --------------------------------------------------------------------------
@pytest.mark.parametrize("factory", [P.single_gauss, P.bw_gauss, P.collider])
def test_calls_bit_exact_fp64(V, O, factory):
    pr = factory()
    o = O.Oracle(pr)
    g = V.Vamp(pr)
    # adapt a little so that grids and α are not trivial, then copy the state
    for it in range(2):
        o.sample_pass(20_000, it, n_threads=NTHREADS)
        o.refine_grids()
        if pr.adapt_alpha:
            o.update_alpha()
    st = o.get_state()
    g.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    N = 2_000_000
    assert g.allocate(N) == o.allocate(N)
    calls = np.unique(np.concatenate([np.arange(0, 300), np.linspace(0, o.allocate(N) - 1, 300).astype(int)]))
    for mode, field in ((0, 11), (1, 0x80000000 | 3)):
        # eval in runs so that the GPU evaluates contiguous ranges
        for c0 in calls[::50]:
            cnt = 50
            r = g.eval_calls(mode, field, int(c0), cnt)
            for q in range(cnt):
                ref = o.eval_call(mode, field, int(c0) + q)
                assert r["channel"][q] == ref["channel"]
                assert np.array_equal(r["jf"][q], ref["jf"])
                assert np.array_equal(r["bins"][q], ref["bins"]), (mode, int(c0) + q)
                assert rel(r["x"][q], ref["x"]) < 1e-13
                assert rel(r["p"][q], ref["p"]) < 1e-12
                assert rel(r["f"][q], ref["f"]) < 1e-12
                assert rel(r["g"][q], ref["g"]) < 1e-12
                assert rel(r["w"][q], ref["w"]) < 1e-12


# --------------------------------------------------------------------------
# FP64 pass parity over whole adaptation schedules
# --------------------------------------------------------------------------
def test_fp64_schedule_single_gauss(V, O):
    pr = P.single_gauss()
    run_schedule(V, O, pr, pr.iterations, pr.calls)


def test_fp64_schedule_bw_gauss_reduced(V, O):
    pr = P.bw_gauss()
    run_schedule(V, O, pr, pr.iterations, 200_000)


def test_fp64_schedule_collider_reduced(V, O):
    pr = P.collider()
    run_schedule(V, O, pr, 3, 150_007)  # ragged call count


def test_fp64_smoothing_and_second_moment(V, O):
    pr = P.bw_gauss().replace(smooth=1, omega_mode=1, beta=1.0)
    run_schedule(V, O, pr, 4, 50_000)


# --------------------------------------------------------------------------
# full-size pass (the benchmark's launch shape): sampled calls + invariants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_pass_sampled_and_invariants(V, O, prec):
    pr = P.collider()
    g = V.Vamp(pr, precision=prec)
    o = O.Oracle(pr)
    N = pr.calls  # 1e7 calls in one pass
    r = g.sample_pass(N, 0)
    assert r.n_calls == o.allocate(N)
    ps = g.get_pass()
    # every axis of a channel sees every call of the channel once: the row
    # sums of D equal Σ w² of the channel (shift 0 on the first pass)
    rows = ps["D"].sum(axis=2)
    Wc = (ps["Vc"] * (ps["Nc"] - 1) / ps["Nc"] + ps["Ic"] ** 2) * ps["Nc"]
    np.testing.assert_allclose(rows, np.repeat(Wc[:, None], pr.d, 1), rtol=1e-9)
    assert abs(r.integral - np.sum(g.get_state()["alpha"] * ps["Ic"])) <= 1e-12 * r.integral
    # sampled calls of this very pass recomputed one by one by the oracle
    idx = np.linspace(0, r.n_calls - 1, 40).astype(np.int64)
    tolw = 1e-12 if prec == 0 else 2e-3
    nbad = 0
    for c0 in idx:
        rg = g.eval_calls(0, 0, int(c0), 1)
        ro = o.eval_call(0, 0, int(c0))
        assert rg["channel"][0] == ro["channel"]
        assert np.array_equal(rg["jf"][0], ro["jf"])
        if rel(rg["w"][0], ro["w"]) >= tolw:
            nbad += 1
    assert nbad == 0 if prec == 0 else nbad <= 2
    # w_max is the maximum of the weights: no sampled weight exceeds it
    assert r.w_max > 0 and r.efficiency == pytest.approx(r.integral / r.w_max, rel=1e-15)


# --------------------------------------------------------------------------
# FP32-eval accuracy against the FP64 oracle on the same state
# --------------------------------------------------------------------------
def test_fp32_eval_pass_accuracy(V, O):
    pr = P.collider()
    o = O.Oracle(pr)
    for it in range(2):
        o.sample_pass(100_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    g32 = V.Vamp(pr, precision=1)
    g32.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    N = 1_000_000
    r32 = g32.sample_pass(N, 7)
    ro = o.sample_pass(N, 7, n_threads=NTHREADS)
    sig = math.sqrt(ro.variance)
    err = abs(r32.integral - ro.integral)
    print(f"\nFP32-eval integral {r32.integral:.12g} oracle {ro.integral:.12g} rel {err / ro.integral:.3e} "
          f"sigma-frac {err / sig:.3e}")
    assert err / ro.integral < 1e-6
    assert err < 0.05 * sig
    assert abs(math.sqrt(r32.variance) / sig - 1) < 1e-3


def test_fp32_eval_per_call_weights(V, O):
    pr = P.collider()
    o = O.Oracle(pr)
    o.sample_pass(100_000, 0, n_threads=NTHREADS)
    o.refine_grids()
    o.update_alpha()
    st = o.get_state()
    g32 = V.Vamp(pr, precision=1)
    g32.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    Nt = g32.allocate(1_000_000)
    assert Nt == o.allocate(1_000_000)
    r = g32.eval_calls(0, 5, 0, 2000)
    relw, flips = [], 0
    for q in range(2000):
        ref = o.eval_call(0, 5, q)
        assert r["channel"][q] == ref["channel"]
        assert np.array_equal(r["jf"][q], ref["jf"])  # forward bins: integer arithmetic
        flips += int(np.sum(r["bins"][q] != ref["bins"]))
        relw.append(abs(r["w"][q] / ref["w"] - 1))
    relw = np.array(relw)
    print(f"\nFP32-eval per-call |dw/w|: median {np.median(relw):.2e} p99 {np.quantile(relw, 0.99):.2e} "
          f"max {relw.max():.2e}; inverse-lookup bin flips {flips} of {2000 * pr.n_channels * pr.d}")
    assert np.median(relw) < 1e-5
    assert flips <= 2000 * pr.n_channels * pr.d * 1e-3


# --------------------------------------------------------------------------
# generation: same events, same order, same counters as the oracle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("factory", [P.bw_gauss, P.collider])
def test_generation_bit_exact_fp64(V, O, factory):
    import torch
    pr = factory().replace(gen_batch=1 << 14)
    o = O.Oracle(pr)
    for it in range(3):
        o.sample_pass(50_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    wm = 0.5 * st["w_max"]  # force overweights and between-batch raises
    o.set_state(w_max=wm, have_pass=True)
    g = V.Vamp(pr)
    g.set_state(st["edges"], st["alpha"], st["shift"], wm)
    n_ev = 600 if pr.n_channels > 8 else 3000
    p, w, stats = g.generate_torch(n_ev, gen_id=2)
    ref = o.generate(n_ev, gen_id=2)
    assert stats["n_written"] == ref["n_written"] == n_ev
    assert stats["n_calls_used"] == ref["n_calls_used"]
    assert stats["n_overweight"] == ref["n_overweight"]
    np.testing.assert_array_equal(p, ref["p"])
    assert rel(w, ref["w"]) < 1e-12
    assert rel(g.get_state()["w_max"], o.get_state()["w_max"]) < 1e-12
    torch.cuda.synchronize()


def test_generation_zero_events_and_errors(V, O):
    import torch
    pr = P.bw_gauss()
    g = V.Vamp(pr)
    buf = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(V.VampError) as e:
        g.generate(10, buf.data_ptr())
    assert e.value.status == V.VAMP_ERR_STATE
    with pytest.raises(V.VampError) as e:
        g.refine_grids()
    assert e.value.status == V.VAMP_ERR_STATE
    g.sample_pass(10_000, 0)
    assert g.generate(0, 0)["n_written"] == 0
    with pytest.raises(V.VampError) as e:
        g.generate(10, buf.data_ptr() + 4)  # misaligned
    assert e.value.status == V.VAMP_ERR_INVALID_ARG
    with pytest.raises(V.VampError) as e:
        g.sample_pass(10, 1 << 31)
    assert e.value.status == V.VAMP_ERR_INVALID_ARG


# --------------------------------------------------------------------------
# edge cases of the shapes
# --------------------------------------------------------------------------
def _edge_problem(d, n, K, seed=9):
    rng = np.random.default_rng(seed)
    ms = P.MapSet.identity(K)
    for c in range(K):
        if d >= 1 and c % 2 == 1:
            ms.n_mapped[c] = 1
            ms.coord[c, 0] = int(rng.integers(0, d))
            ms.kind[c, 0] = P.MAP_BW if c % 4 == 1 else P.MAP_POW
            ms.a[c, 0] = 0.4
            ms.b[c, 0] = 5e-3
    w = rng.exponential(1.0, K)
    return P.Problem(name=f"edge_{d}_{n}_{K}", d=d, n_bins=n, channels=ms, peak_weight=w / w.sum(),
                     peaks=ms.copy(), gauss_sigma=0.2, gauss_centre=0.5, gauss_norm=P.GAUSS_NORM_UNIT,
                     seed=seed, iterations=3, calls=3000, adapt_grid=True, adapt_alpha=True)


@pytest.mark.parametrize("d,n,K,calls", [
    (1, 1, 1, 1),        # one bin, one call (N_min applies)
    (1, 2, 3, 37),
    (16, 256, 2, 5003),  # largest dimension and bin count
    (3, 7, 33, 4099),    # ragged everything
    (16, 100, 64, 20000),
])
def test_edge_shapes_fp64(V, O, d, n, K, calls):
    run_schedule(V, O, _edge_problem(d, n, K), 3, calls)


def test_switched_off_channel(V, O):
    pr = P.bw_gauss()
    o = O.Oracle(pr)
    g = V.Vamp(pr)
    a = np.array([0.3, 0.0, 0.2, 0.0, 0.25, 0.25])
    st = o.get_state()
    o.set_state(alpha=a, have_pass=True)
    g.set_state(st["edges"], a, st["shift"], 0.0)
    rg = g.sample_pass(30_000, 4)
    ro = o.sample_pass(30_000, 4, n_threads=NTHREADS)
    assert rg.n_calls == ro.n_calls and rel(rg.integral, ro.integral) < 1e-12
    assert list(g.get_pass()["Nc"][[1, 3]]) == [0, 0]
    g.update_alpha()
    o.update_alpha()
    assert rel(g.get_state()["alpha"], o.get_state()["alpha"]) < 1e-12


def test_repeatable(V):
    pr = P.collider()
    a = V.Vamp(pr).sample_pass(500_000, 3)
    b = V.Vamp(pr).sample_pass(500_000, 3)
    assert abs(a.integral - b.integral) <= 1e-13 * a.integral
    assert a.w_max == b.w_max


def test_contexts_with_different_shapes_coexist(V, O):
    """A context with a larger shared-memory need, created first, still runs
    after a smaller one was created (the kernel limit is only raised)."""
    big = V.Vamp(_edge_problem(16, 256, 8), precision=1)
    small = V.Vamp(P.single_gauss(), precision=1)
    rb = big.sample_pass(20_000, 0)
    rs = small.sample_pass(10_000, 0)
    assert rb.n_calls > 0 and rs.n_calls == 10_000


# --------------------------------------------------------------------------
# FP64 power-law maps: the inverse fifth root by Newton's method against the
# oracle's pow() (libm), over the exponent range the range reduction spans
# --------------------------------------------------------------------------
def test_fp64_power_maps_match_libm_pow(V, O):
    """Channels mapping by x^5 with δ = 0, 1e-3 and 5 (so p + δ spans
    [2^-1022, 6]); per-call bins bit-exact, coordinates, g, f and weights
    within 1e-13 of the oracle, whose maps call pow()."""
    ms = P.MapSet.identity(3)
    for c, dl in enumerate((0.0, 1e-3, 5.0)):
        ms.n_mapped[c] = 1
        ms.coord[c, 0] = c
        ms.kind[c, 0] = P.MAP_POW
        ms.b[c, 0] = dl
    pr = P.Problem(name="pow3", d=3, n_bins=30, channels=ms, peak_weight=np.array([0.5, 0.3, 0.2]),
                   peaks=ms.copy(), gauss_sigma=0.2, gauss_centre=0.5, gauss_norm=P.GAUSS_NORM_UNIT, seed=4,
                   iterations=3, calls=20_000, adapt_grid=True, adapt_alpha=True)
    o = O.Oracle(pr)
    for it in range(2):
        o.sample_pass(20_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    g = V.Vamp(pr)
    g.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    assert g.allocate(100_000) == o.allocate(100_000)
    r = g.eval_calls(0, 3, 0, 3000)
    worst = 0.0
    for q in range(3000):
        ref = o.eval_call(0, 3, q)
        assert np.array_equal(r["bins"][q], ref["bins"]), q
        for key in ("x", "p"):
            assert rel(r[key][q], ref[key]) < 1e-13, (key, q)
        for key in ("f", "g", "w"):
            worst = max(worst, rel(r[key][q], ref[key]))
    print(f"\nFP64 power-law maps: largest relative deviation of f, g, w from the oracle {worst:.2e}")
    assert worst < 1e-13

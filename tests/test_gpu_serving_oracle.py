"""The request loop (vamp_server_*) and FP32-eval generation against the
FP64 oracle.

1. A staggered mix of requests of uneven shape (the serving workload's
   recipe: d, channels, bins and calls drawn per request) is served by the
   FP64 server while later requests keep arriving; every request is then
   replayed by the oracle on its own -- the same iterations of calls, the
   rebinning (Eq. 14) and α update (Eq. 25) after each, passes combined from
   combine_from on, then its events from generation stream 0 (§2 Eq. 2, §3.5
   on unweighting) -- and compared: last pass, combination and grids within
   1e-12, events bit-exact.

2. FP32-eval generation on the adapted collider state: with the oracle's
   random stream the accepted events are the oracle's up to the rare accept
   decisions that FP32 rounding flips; on independent streams the acceptance
   rates agree within their binomial errors and every coordinate's marginal
   passes a two-sample Kolmogorov-Smirnov test against the oracle's events.
"""
import math
import os
import time

import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _requests(n, seed=21):
    out = []
    for i, rq in enumerate(P.serving_stream(rate_per_s=1000.0, duration_s=10.0, seed=seed, max_requests=n)):
        pr = rq.problem.replace(gen_batch=1 << 15)
        iters = 2 + i % 4  # 2..5 iterations; passes combined from iteration pr.combine_from on
        out.append((pr, iters, max(20_000, pr.calls // 20), min(pr.n_events, 1000)))
    return out


def _oracle_run(O, pr, iters, calls, n_ev):
    o = O.Oracle(pr)
    r = None
    for it in range(iters):
        r = o.sample_pass(calls, it, combine=it >= pr.combine_from, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    ev = o.generate(n_ev, gen_id=0) if n_ev else None
    return r, o.get_state(), ev


def test_served_requests_equal_the_oracle(oracle_mod):
    import torch
    from paper_1811_09711_gb300 import vamp as V
    reqs = _requests(10)
    srv = V.Server(max_slots=4, mem_budget_bytes=8 << 30, precision=V.PREC_FP64)
    bufs, states, ids = [], [], []
    for i, (pr, iters, calls, n_ev) in enumerate(reqs):
        buf = torch.zeros(max(1, n_ev) * V.record_bytes(pr.d), dtype=torch.uint8, device="cuda")
        sbuf = torch.full((pr.n_channels * pr.d * (pr.n_bins + 1) + 2 * pr.n_channels,), -1.0,
                          dtype=torch.float64, device="cuda")
        bufs.append(buf)
        states.append(sbuf)
        torch.cuda.synchronize()
        ids.append(srv.submit(pr, iters, calls, n_ev, buf.data_ptr(), state_ptr=sbuf.data_ptr()))
        if i % 3 == 2:
            time.sleep(0.02)  # later requests arrive while earlier ones are in flight
    srv.wait_idle(600.0)
    done = {r.id: r for r in srv.poll(len(reqs) + 4)}
    stats = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    assert sorted(done) == sorted(ids)
    assert stats["mem_in_use"] == 0
    queued = sum(done[i].queue_s > 0.0 for i in ids)
    assert queued > 0  # more requests than slots: some waited for a slot
    for rid, buf, sbuf, (pr, iters, calls, n_ev) in zip(ids, bufs, states, reqs):
        r = done[rid]
        assert r.status == V.VAMP_OK and r.iterations == iters, pr.name
        ro, so, evo = _oracle_run(oracle_mod, pr, iters, calls, n_ev)
        res = r.result
        assert res.n_calls == ro.n_calls, pr.name
        assert _rel(res.integral, ro.integral) < 1e-12, (pr.name, res.integral, ro.integral)
        m2 = ro.variance + ro.integral ** 2 / ro.n_calls
        assert abs(res.variance - ro.variance) <= 1e-12 * m2, pr.name
        # w_max is one call's weight: a last-bit difference in a Breit-Wigner
        # argument near the pole of tan is amplified, so it gets a looser bar
        assert _rel(res.w_max, ro.w_max) < 1e-10, pr.name
        if iters - 1 >= pr.combine_from:
            assert _rel(res.combined, ro.combined) < 1e-12, pr.name
            assert _rel(res.combined_sigma, ro.combined_sigma) < 1e-12, pr.name
        K, d, n = pr.n_channels, pr.d, pr.n_bins
        st = sbuf.cpu().numpy()
        ne = K * d * (n + 1)
        # each rebinning agrees within 1e-12 (as in the per-iteration schedule
        # tests); over `iters` rebinnings the differences can add up
        np.testing.assert_allclose(st[:ne].reshape(K, d, n + 1), so["edges"], rtol=0, atol=1e-12 * iters)
        np.testing.assert_allclose(st[ne:ne + K], so["alpha"], rtol=1e-10, atol=0)
        assert r.events_written == n_ev
        if n_ev:
            p_s, w_s = V.decode_records(buf[: n_ev * V.record_bytes(d)].cpu().numpy(), d)
            assert evo["n_written"] == n_ev
            assert r.events_calls_used == evo["n_calls_used"], pr.name
            assert r.events_overweight == evo["n_overweight"], pr.name
            np.testing.assert_array_equal(p_s, evo["p"])
            # a weight is f over a product of d bin densities 1/(n dx): grids
            # that differ by de move each density by at most 2 de / dx
            e_g = st[:ne].reshape(K, d, n + 1)
            de = float(np.max(np.abs(e_g - so["edges"])))
            dx = float(np.min(np.diff(so["edges"], axis=2)))
            np.testing.assert_allclose(w_s, evo["w"], rtol=1e-12 + 2 * d * de / dx)


@pytest.fixture(scope="module")
def collider_state(oracle_mod):
    pr = P.collider().replace(gen_batch=1 << 18)
    o = oracle_mod.Oracle(pr)
    for it in range(4):
        o.sample_pass(1_000_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    return pr, o, o.get_state()


@pytest.mark.parametrize("family", ["k_union", "k_pass"])
def test_fp32_generation_against_oracle(oracle_mod, collider_state, family):
    """FP32-eval generation by each kernel family (union tables and staged
    tiles) against the oracle's events on the collider."""
    from scipy import stats
    from paper_1811_09711_gb300 import vamp as V
    pr, o, st = collider_state
    n_ev = 6000
    g = V.Vamp(pr, precision=V.PREC_FP32_EVAL)
    g.select_family(family)
    g.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    # same random stream: the oracle's events up to flipped accept decisions
    p_g, w_g, s_g = g.generate_torch(n_ev, gen_id=3)
    assert g.kernel_name(1).startswith(family + "<float, 1,"), g.kernel_name(1)
    o.set_state(w_max=st["w_max"], have_pass=True)
    ev_o = o.generate(n_ev, gen_id=3)
    assert s_g["n_written"] == ev_o["n_written"] == n_ev
    used_g, used_o = s_g["n_calls_used"], ev_o["n_calls_used"]
    assert abs(used_g - used_o) <= max(2, 1e-3 * used_o), (used_g, used_o)
    d = np.abs(p_g[:, None, :].astype(np.float64) - ev_o["p"][None, :, :].astype(np.float64)).max(axis=2)
    near = float((d.min(axis=1) <= 1e-5).mean())
    print(f"\nFP32-eval events on the oracle's stream: {near:.4f} matched, calls {used_g} vs {used_o}")
    assert near >= 0.99
    # independent streams: acceptance rates and marginals
    g2 = V.Vamp(pr, precision=V.PREC_FP32_EVAL)
    g2.select_family(family)
    g2.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    p2, _, s2 = g2.generate_torch(n_ev, gen_id=11)
    o.set_state(w_max=st["w_max"], have_pass=True)
    e2 = o.generate(n_ev, gen_id=12)
    r_g, r_o = n_ev / s2["n_calls_used"], n_ev / e2["n_calls_used"]
    se = math.sqrt(r_g * (1 - r_g) / s2["n_calls_used"] + r_o * (1 - r_o) / e2["n_calls_used"])
    print(f"acceptance FP32-eval {r_g:.5f}, oracle {r_o:.5f} (difference {abs(r_g - r_o) / se:.2f} sigma)")
    assert abs(r_g - r_o) < 4 * se
    pmin = 1.0
    for k in range(pr.d):
        pv = stats.ks_2samp(p2[:, k], e2["p"][:, k]).pvalue
        pmin = min(pmin, pv)
    print(f"smallest KS p-value over the {pr.d} marginals: {pmin:.3g}")
    # 14 tests at level 1e-3 each: a false alarm has probability < 1.4 %
    assert pmin > 1e-3

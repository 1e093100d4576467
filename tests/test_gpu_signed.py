"""Integrands of both signs (§3.1; reading R19) on the GPU against the FP64
oracle, through the C ABI: adaptation runs within 1e-12 in FP64, generation
bit-exact (accept with |w|, records keep the sign, w_max raised to the
largest |w|), the FP32-eval pass within its tolerance, batches equal to
contexts."""
import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P
from test_gpu_parity import NTHREADS, rel, run_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1811_09711_gb300 import vamp
    return vamp


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


@pytest.mark.parametrize("factory,calls", [(lambda: P.signed_pair(d=2), 40_000),
                                           (lambda: P.signed_pair(weights=(-1.3, 0.3), d=3), 40_000),
                                           (P.signed_bw_gauss, 300_000)])
def test_signed_schedule_fp64(V, O, factory, calls):
    pr = factory().replace(combine_from=1)
    _, _, out = run_schedule(V, O, pr, 4, calls)
    assert min(ro.integral for _, ro in out) != 0.0


@pytest.mark.parametrize("weights", [(1.3, -0.3), (-1.3, 0.3)])
def test_signed_generation_bit_exact_fp64(V, O, weights):
    import torch
    pr = P.signed_pair(weights=weights, d=2).replace(gen_batch=1 << 12)
    o = O.Oracle(pr)
    for it in range(3):
        o.sample_pass(30_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    wm = 0.3 * st["w_max"]  # overweights and between-batch raises
    o.set_state(w_max=wm, have_pass=True)
    g = V.Vamp(pr)
    g.set_state(st["edges"], st["alpha"], st["shift"], wm)
    n_ev = 5000
    p, w, stats = g.generate_torch(n_ev, gen_id=4)
    ref = o.generate(n_ev, gen_id=4)
    torch.cuda.synchronize()
    assert stats["n_written"] == ref["n_written"] == n_ev
    assert stats["n_calls_used"] == ref["n_calls_used"]
    assert stats["n_overweight"] == ref["n_overweight"] > 0
    np.testing.assert_array_equal(p, ref["p"])
    assert np.array_equal(np.sign(w), np.sign(ref["w"])) and (w < 0).any() and (w > 0).any()
    assert rel(w, ref["w"]) < 1e-12
    assert rel(g.get_state()["w_max"], o.get_state()["w_max"]) < 1e-12


def test_signed_fp32_eval_accuracy(V, O):
    """Same grids and random stream: the FP32-eval pass is within 1e-6 of the
    scale Σ|w_q| of the integrand and 0.05σ of the FP64 oracle."""
    pr = P.signed_bw_gauss()
    o = O.Oracle(pr)
    for it in range(3):
        o.sample_pass(300_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    g = V.Vamp(pr, precision=1)
    g.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    rg = g.sample_pass(2_000_000, 3)
    ro = o.sample_pass(2_000_000, 3, n_threads=NTHREADS)
    scale = float(np.abs(pr.peak_weight).sum())
    assert rg.n_calls == ro.n_calls
    assert abs(rg.integral - ro.integral) < 1e-6 * scale
    assert abs(rg.integral - ro.integral) < 0.05 * np.sqrt(ro.variance)
    assert rel(rg.w_max, ro.w_max) < 1e-5


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_signed_in_batch_equals_alone(V, precision, tol):
    probs = [P.signed_pair(d=2).replace(calls=30_000), P.signed_bw_gauss().replace(calls=100_000),
             P.signed_pair(weights=(-1.3, 0.3), d=4).replace(calls=30_000)]
    batch = V.Batch(probs, precision=precision, autotune=False)
    alone = [V.Vamp(pr, precision=precision) for pr in probs]
    for g in alone:
        g.select_family("k_pass")  # the FP32-eval arithmetic of the batch kernel
    for it in range(3):
        rb = batch.iterate([pr.calls for pr in probs], it, adapt=3)
        for i, (pr, g) in enumerate(zip(probs, alone)):
            ra = g.sample_pass(pr.calls, it)
            g.refine_grids()
            g.update_alpha()
            assert rb[i].n_calls == ra.n_calls
            assert abs(rb[i].integral - ra.integral) <= tol * abs(ra.integral), (i, it)
            assert rel(rb[i].w_max, ra.w_max) < 1e3 * tol

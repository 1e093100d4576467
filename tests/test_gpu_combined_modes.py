"""Pseudo-stratified sampling, channel equivalences and an integrand of both
signs together (§3.3, §3.5, §3.1), GPU against the FP64 oracle: whole FP64
adaptation runs within 1e-12, the FP32-eval pass within 1e-6 of the scale of
the integrand and 0.05σ."""
import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P
from test_gpu_parity import NTHREADS, run_schedule

pytestmark = pytest.mark.gpu


def _problem():
    pr = P.ring(3, 5, kind=P.EQ_SYMMETRIC)
    w = np.array([1.4, -0.6, 0.2])  # peak of channel 1 negative: f < 0 near its resonance
    return pr.replace(peak_weight=w, stratified=1, combine_from=1, n_bins=16)


@pytest.fixture(scope="module")
def V():
    from paper_1811_09711_gb300 import vamp
    return vamp


def test_combined_modes_schedule_fp64(V, oracle_mod):
    run_schedule(V, oracle_mod, _problem(), 4, 60_000)


def test_combined_modes_fp32_eval(V, oracle_mod):
    pr = _problem()
    o = oracle_mod.Oracle(pr)
    for it in range(3):
        o.sample_pass(100_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    g = V.Vamp(pr, precision=1)
    g.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    rg = g.sample_pass(1_000_000, 3)
    ro = o.sample_pass(1_000_000, 3, n_threads=NTHREADS)
    assert rg.n_calls == ro.n_calls
    scale = float(np.abs(pr.peak_weight).sum())
    assert abs(rg.integral - ro.integral) < 1e-6 * scale
    assert abs(rg.integral - ro.integral) < 0.05 * np.sqrt(ro.variance)

"""Many uneven integrations in one persistent launch (vamp_batch_*), GPU.

* every instance's pass results, grids and α equal those of the same
  instance run alone through vamp_create (same random streams), within the
  tolerance of the precision: 1e-12 relative for FP64, 1e-9 for FP32-eval
  (the two paths may round single calls differently in the last bit);
* an FP64 batch matches the FP64 oracle instance by instance (1e-12).
"""
import os

import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def _instances(n, scale=200, first=0):
    out = []
    for i in range(first, first + n):
        pr = P.batch_instance(i)
        out.append(pr.replace(calls=max(2000, pr.calls // scale)))
    return out


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_batch_equals_alone(precision, tol):
    from paper_1811_09711_gb300 import vamp as V
    probs = _instances(14)
    batch = V.Batch(probs, precision=precision, autotune=True)
    alone = [V.Vamp(pr, precision=precision) for pr in probs]
    for g in alone:
        g.select_family("k_pass")  # the FP32-eval arithmetic of the batch kernel
    worst = 0.0
    for it in range(3):
        ncalls = [pr.calls for pr in probs]
        rb = batch.iterate(ncalls, it, adapt=3)
        for i, (pr, g) in enumerate(zip(probs, alone)):
            ra = g.sample_pass(ncalls[i], it)
            g.refine_grids()
            g.update_alpha()
            assert rb[i].n_calls == ra.n_calls, (i, it)
            worst = max(worst, _rel(rb[i].integral, ra.integral))
            assert _rel(rb[i].integral, ra.integral) < tol, (i, it, rb[i].integral, ra.integral)
            assert _rel(rb[i].w_max, ra.w_max) < tol
            sb, sa = batch.get_state(i), g.get_state()
            np.testing.assert_allclose(sb["edges"], sa["edges"], rtol=0, atol=1e3 * tol)
    print(f"\nbatch vs alone, worst relative integral difference: {worst:.2e}")
    t = batch.tuning()
    assert t["item_calls"] % 256 == 0 and t["budget_kb"] in (72, 112)


def test_batch_fp64_matches_oracle(oracle_mod):
    from paper_1811_09711_gb300 import vamp as V
    probs = _instances(5, scale=400, first=20)
    batch = V.Batch(probs, precision=0, autotune=False)
    orcs = [oracle_mod.Oracle(pr) for pr in probs]
    for it in range(2):
        rb = batch.iterate([pr.calls for pr in probs], it, adapt=3)
        for i, (pr, o) in enumerate(zip(probs, orcs)):
            ro = o.sample_pass(pr.calls, it, combine=it >= pr.combine_from, n_threads=NTHREADS)
            o.refine_grids()
            o.update_alpha()
            assert rb[i].n_calls == ro.n_calls
            assert _rel(rb[i].integral, ro.integral) < 1e-12, (i, it)
            np.testing.assert_allclose(batch.get_state(i)["edges"], o.get_state()["edges"], rtol=0, atol=1e-12)


def test_batch_rejects_bad_input():
    from paper_1811_09711_gb300 import vamp as V
    probs = _instances(3)
    batch = V.Batch(probs, precision=1, autotune=False)
    with pytest.raises(V.VampError):
        batch.iterate([0, 10, 10], 0)
    with pytest.raises(V.VampError):
        batch.iterate([10, 10, 10], 1 << 31)
    r = batch.iterate([1000, 1000, 1000], 0)
    # N' = Σ max(N_min, floor(α_c N)) lies within K of N from below and K N_min above
    for x, pr in zip(r, probs):
        assert 1000 - pr.n_channels <= x.n_calls <= 1000 + pr.n_channels * pr.n_min

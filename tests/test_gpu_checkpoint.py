"""Checkpoint / restore of the adaptation state (grids, α, shifts, w_max and
the pass history of the iteration combination): a run interrupted after
iteration 3, restored into a new context and continued equals the
uninterrupted run (up to the order of FP64 atomic sums); a checkpoint of
another shape is rejected."""
import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu


def _iterate(g, n, it0, iters):
    r = None
    for it in range(it0, it0 + iters):
        r = g.sample_pass(n, it)
        g.refine_grids()
        g.update_alpha()
    return r


def _modes_problem():
    """Pseudo-stratified, with symmetric channel equivalences and a peak of
    negative weight."""
    return P.ring(3, 5, kind=P.EQ_SYMMETRIC).replace(peak_weight=np.array([1.4, -0.6, 0.2]), stratified=1,
                                                      combine_from=1, n_bins=16)


@pytest.mark.parametrize("precision,tol,factory", [(0, 1e-12, "bw_gauss"), (1, 1e-9, "bw_gauss"),
                                                   (0, 1e-12, "modes")])
def test_restored_run_continues_the_uninterrupted_run(precision, tol, factory):
    from paper_1811_09711_gb300 import vamp as V
    pr = P.bw_gauss().replace(combine_from=1) if factory == "bw_gauss" else _modes_problem()
    n = 100_000
    full = V.Vamp(pr, precision=precision)
    rf = _iterate(full, n, 0, 5)
    first = V.Vamp(pr, precision=precision)
    _iterate(first, n, 0, 3)
    blob = first.checkpoint()
    del first
    resumed = V.Vamp(pr, precision=precision)
    resumed.restore(blob)
    rr = _iterate(resumed, n, 3, 2)
    for k in ("integral", "variance", "w_max", "combined", "combined_sigma", "chi2_dof"):
        a, b = getattr(rr, k), getattr(rf, k)
        assert abs(a - b) <= tol * max(abs(b), 1e-300), (k, a, b)
    sf, sr = full.get_state(), resumed.get_state()
    np.testing.assert_allclose(sr["edges"], sf["edges"], rtol=0, atol=tol)
    np.testing.assert_allclose(sr["alpha"], sf["alpha"], rtol=tol, atol=0)


def test_restore_rejects_other_shapes_and_garbage():
    from paper_1811_09711_gb300 import vamp as V
    g = V.Vamp(P.bw_gauss(), precision=1)
    _iterate(g, 20_000, 0, 1)
    blob = g.checkpoint()
    other = V.Vamp(P.single_gauss(), precision=1)
    with pytest.raises(V.VampError):
        other.restore(blob)
    with pytest.raises(V.VampError):
        g.restore(b"not a checkpoint at all, really" * 4)
    with pytest.raises(V.VampError):
        g.restore(blob[: len(blob) // 2])
    g.restore(blob)  # the context is still usable
    g.sample_pass(20_000, 1)

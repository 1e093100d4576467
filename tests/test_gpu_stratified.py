"""Pseudo-stratified sampling in r space (§3.3) on the GPU against the FP64
oracle: the cells, forward bins and per-call values bit-exact / 1e-12,
whole adaptation runs (integral, stratified variance, D, edges, α) within
1e-12 in FP64, the FP32-eval form within its tolerance; instances of a batch
and requests of a server equal the same problems alone (and the oracle); the
allocation-free pass rejects the mode."""
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


@pytest.mark.parametrize("factory,calls", [(P.single_gauss, 60_000), (P.bw_gauss, 300_000)])
def test_stratified_schedule_fp64(V, O, factory, calls):
    pr = factory().replace(stratified=1, combine_from=1)
    o = O.Oracle(pr)
    N = o.allocate(calls)
    assert N < calls  # whole cells: the remainder is not sampled
    run_schedule(V, O, pr, 3, calls)


def test_stratified_calls_bit_exact_fp64(V, O):
    pr = P.bw_gauss().replace(stratified=1)
    o = O.Oracle(pr)
    g = V.Vamp(pr)
    for it in range(2):
        o.sample_pass(200_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    g.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    N = 500_000
    assert g.allocate(N) == o.allocate(N)
    n_tot = o.allocate(N)
    for c0 in list(range(0, 400, 50)) + list(np.linspace(0, n_tot - 50, 8).astype(int)):
        r = g.eval_calls(0, 7, int(c0), 50)
        for q in range(50):
            ref = o.eval_call(0, 7, int(c0) + q)
            assert r["channel"][q] == ref["channel"]
            assert np.array_equal(r["jf"][q], ref["jf"]), int(c0) + q
            assert np.array_equal(r["bins"][q], ref["bins"])
            assert rel(r["x"][q], ref["x"]) < 1e-13
            assert rel(r["w"][q], ref["w"]) < 1e-12


def test_stratified_context_after_a_tuned_importance_context(V, O):
    """The kernel choice cached for an importance-sampled context of the same
    shape and call count is not reused for a pseudo-stratified one (whose
    candidates are the generic kernels with the cell code)."""
    pr = P.bw_gauss()
    V.Vamp(pr, precision=1).sample_pass(50_000, 0)  # tunes (and caches) the shape-specialised kernel
    g = V.Vamp(pr.replace(stratified=1), precision=1)
    r = g.sample_pass(50_000, 0)
    assert g.kernel_info()["shape_d"] == 0
    ro = O.Oracle(pr.replace(stratified=1)).sample_pass(50_000, 0, n_threads=NTHREADS)
    assert r.n_calls == ro.n_calls
    assert abs(r.integral - ro.integral) < 0.05 * np.sqrt(ro.variance)


def test_stratified_fp32_eval_accuracy(V, O):
    pr = P.bw_gauss().replace(stratified=1)
    o = O.Oracle(pr)
    g = V.Vamp(pr, precision=1)
    for it in range(2):
        o.sample_pass(300_000, it, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
    st = o.get_state()
    g.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    rg = g.sample_pass(1_000_000, 2)
    ro = o.sample_pass(1_000_000, 2, n_threads=NTHREADS)
    assert rg.n_calls == ro.n_calls
    assert rel(rg.integral, ro.integral) < 1e-6
    assert abs(rg.integral - ro.integral) < 0.05 * np.sqrt(ro.variance)
    assert rel(rg.variance, ro.variance) < 1e-3


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_stratified_instances_in_a_batch_equal_alone(V, precision, tol):
    """Pseudo-stratified and importance-sampled instances in one persistent
    launch give what each gives alone; the second call count is larger than
    the first, so the instances' cell-sum buffers grow between iterations."""
    probs = [P.bw_gauss().replace(stratified=1), P.single_gauss().replace(stratified=1),
             P.batch_instance(3), P.ring(3, 5).replace(stratified=1)]
    batch = V.Batch(probs, precision=precision, autotune=False)
    alone = [V.Vamp(pr, precision=precision) for pr in probs]
    for g in alone:
        g.select_family("k_pass")  # the FP32-eval arithmetic of the batch kernel
    for it, calls in enumerate((40_000, 40_000, 120_000)):
        rb = batch.iterate([calls] * len(probs), it, adapt=3)
        for i, g in enumerate(alone):
            ra = g.sample_pass(calls, it)
            g.refine_grids()
            g.update_alpha()
            assert rb[i].n_calls == ra.n_calls, (i, it)
            assert abs(rb[i].integral - ra.integral) <= tol * abs(ra.integral), (i, it)
            m2 = ra.variance + ra.integral ** 2 / ra.n_calls
            assert abs(rb[i].variance - ra.variance) <= 10 * tol * m2, (i, it)
            np.testing.assert_allclose(batch.get_state(i)["edges"], g.get_state()["edges"], rtol=0,
                                       atol=1e3 * tol)


def test_stratified_batch_matches_oracle_fp64(V, O):
    pr = P.bw_gauss().replace(stratified=1, combine_from=1)
    batch = V.Batch([pr, P.single_gauss().replace(stratified=1)], precision=0, autotune=False)
    o = O.Oracle(pr)
    for it in range(3):
        rb = batch.iterate([100_000, 20_000], it, adapt=3)
        ro = o.sample_pass(100_000, it, combine=True, n_threads=NTHREADS)
        o.refine_grids()
        o.update_alpha()
        assert rb[0].n_calls == ro.n_calls
        assert rel(rb[0].integral, ro.integral) < 1e-12
        m2 = ro.variance + ro.integral ** 2 / ro.n_calls
        assert abs(rb[0].variance - ro.variance) <= 1e-12 * m2
        np.testing.assert_allclose(batch.get_state(0)["edges"], o.get_state()["edges"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_stratified_requests_in_a_server_equal_alone(V, precision, tol):
    """Pseudo-stratified requests served in a mix with an importance-sampled
    one give what each gives alone."""
    import torch
    reqs = [(P.bw_gauss().replace(stratified=1, combine_from=1), 3, 60_000),
            (P.batch_instance(7), 2, 30_000),
            (P.single_gauss().replace(stratified=1, combine_from=1), 4, 20_000)]
    srv = V.Server(max_slots=4, precision=precision)
    ids = [srv.submit(pr, iters, calls, 0, 0) for pr, iters, calls in reqs]
    srv.wait_idle(300.0)
    done = {r.id: r for r in srv.poll(8)}
    srv.close()
    for rid, (pr, iters, calls) in zip(ids, reqs):
        g = V.Vamp(pr, precision=precision)
        g.select_family("k_pass")  # the FP32-eval arithmetic of the server's multi-instance kernel
        for it in range(iters):
            ra = g.sample_pass(calls, it)
            g.refine_grids()
            g.update_alpha()
        torch.cuda.synchronize()
        r = done[rid]
        assert r.status == V.VAMP_OK and r.result.n_calls == ra.n_calls
        assert abs(r.result.integral - ra.integral) <= tol * abs(ra.integral), pr.name
        m2 = ra.variance + ra.integral ** 2 / ra.n_calls
        assert abs(r.result.variance - ra.variance) <= 10 * tol * m2, pr.name


def test_static_pass_rejects_stratified(V):
    import torch
    pr = P.bw_gauss().replace(stratified=1)
    st = V.Vamp(pr.replace(stratified=0)).get_state()
    e = torch.tensor(st["edges"], dtype=torch.float64, device="cuda")
    a = torch.tensor(st["alpha"], dtype=torch.float64, device="cuda")
    s = torch.tensor(st["shift"], dtype=torch.float64, device="cuda")
    with pytest.raises(V.VampError):
        V.sample_pass_static(pr, 1, e.data_ptr(), a.data_ptr(), s.data_ptr(), 10_000, 0)

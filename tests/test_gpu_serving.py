"""Continuous-batching request loop (vamp_server_*), GPU.

Requests arrive while others are being served, wait for a slot, join the
next scheduler tick and leave when done.  Each request's result must not
depend on the mix it was served in: its last pass, its running combination
and its unweighted events equal those of the same request run alone through
vamp_create / sample_pass / refine_grids / update_alpha / generate(gen_id 0).
"""
import time

import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu


def _requests(n, seed=11, min_calls=20000, div=20):
    out = []
    for i, rq in enumerate(P.serving_stream(rate_per_s=1000.0, duration_s=10.0, seed=seed, max_requests=n)):
        pr = rq.problem
        iters = 2 + i % 4  # 2..5 iterations; combination from iteration 4 on
        out.append((pr, iters, max(min_calls, pr.calls // div), min(pr.n_events, 1500)))
    return out


def _alone(V, pr, iters, calls, n_ev, precision):
    import torch
    g = V.Vamp(pr, precision=precision)
    g.select_family("k_pass")  # the FP32-eval arithmetic of the server's multi-instance kernel
    r = None
    for it in range(iters):
        r = g.sample_pass(calls, it)
        g.refine_grids()
        g.update_alpha()
    ev = g.generate_torch(n_ev, gen_id=0) if n_ev > 0 else None
    torch.cuda.synchronize()
    return r, ev


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _near_fraction(p_s, p_a, atol=1e-5):
    """Fraction of served events with an event of the alone run within atol
    in every coordinate.  FP32-eval coordinates may differ in the last bits
    where the two kernels round differently, and an accept decision may flip
    and shift the order, so events are matched as sets."""
    if len(p_s) == 0:
        return 1.0
    d = np.abs(p_s[:, None, :].astype(np.float64) - p_a[None, :, :].astype(np.float64)).max(axis=2)
    return float((d.min(axis=1) <= atol).mean())


def _serve(V, reqs, precision, max_slots, budget, stagger, t_sub=None):
    import torch
    srv = V.Server(max_slots=max_slots, mem_budget_bytes=budget, precision=precision)
    bufs, ids = [], []
    for i, (pr, iters, calls, n_ev) in enumerate(reqs):
        buf = torch.zeros(max(1, n_ev) * V.record_bytes(pr.d), dtype=torch.uint8, device="cuda")
        bufs.append(buf)
        torch.cuda.synchronize()
        if t_sub is not None:
            t_sub.append(time.perf_counter())
        ids.append(srv.submit(pr, iters, calls, n_ev, buf.data_ptr()))
        if stagger and i % 3 == 2:
            time.sleep(0.01)  # later requests arrive while earlier ones are in flight
    srv.wait_idle(300.0)
    done = {r.id: r for r in srv.poll(len(reqs) + 8)}
    stats = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    return ids, bufs, done, stats


# w_max is one call's weight, not a mean: where the two kernels round a map
# argument differently in the last bit, the Breit-Wigner inverse (tan near
# its pole) amplifies it, so the maximum gets a looser bound than the sums
@pytest.mark.parametrize("precision,tol,tol_wmax", [(0, 1e-12, 1e-10), (1, 1e-9, 1e-6)])
def test_requests_in_a_mix_equal_requests_alone(precision, tol, tol_wmax):
    from paper_1811_09711_gb300 import vamp as V
    reqs = _requests(12)
    ids, bufs, done, stats = _serve(V, reqs, precision, max_slots=5, budget=8 << 30, stagger=True)
    assert sorted(done) == sorted(ids) and len(set(ids)) == len(ids)
    assert stats["mem_in_use"] == 0
    assert stats["ticks"] >= max(it for _, it, _, _ in reqs)
    assert stats["events"] == sum(n for *_, n in reqs)
    queued = 0
    for rid, buf, (pr, iters, calls, n_ev) in zip(ids, bufs, reqs):
        r = done[rid]
        assert r.status == V.VAMP_OK and r.iterations == iters
        assert 0.0 <= r.queue_s <= r.latency_s
        queued += r.queue_s > 0.0
        ra, ev = _alone(V, pr, iters, calls, n_ev, precision)
        assert r.result.n_calls == ra.n_calls
        assert _rel(r.result.integral, ra.integral) < tol, (pr.name, r.result.integral, ra.integral)
        assert _rel(r.result.w_max, ra.w_max) < tol_wmax, (pr.name, r.result.w_max, ra.w_max)
        assert _rel(r.result.combined, ra.combined) < tol
        assert abs(r.result.chi2_dof - ra.chi2_dof) < 1e3 * tol * max(1.0, abs(ra.chi2_dof))
        assert r.events_written == n_ev
        if n_ev:
            p_a, w_a, st = ev
            assert st["n_written"] == n_ev and r.events_calls_used == st["n_calls_used"]
            p_s, w_s = V.decode_records(buf[: n_ev * V.record_bytes(pr.d)].cpu().numpy(), pr.d)
            if precision == 0:
                np.testing.assert_array_equal(p_s, p_a)
                np.testing.assert_allclose(w_s, w_a, rtol=1e-9)
            else:
                assert _near_fraction(p_s, p_a) >= 0.98, pr.name
    assert queued > 0  # more requests than slots: some waited


def test_budget_admits_one_request_at_a_time():
    """A budget below any request's footprint serves requests one by one
    (a request that alone exceeds the budget runs when nothing else does)."""
    from paper_1811_09711_gb300 import vamp as V
    reqs = _requests(4, seed=12)
    t_sub = []
    ids, bufs, done, stats = _serve(V, reqs, 1, max_slots=8, budget=1, stagger=False, t_sub=t_sub)
    assert stats["mem_in_use"] == 0
    # host times of admission and completion (to within the submit call's duration)
    spans = sorted((t + done[i].queue_s, t + done[i].latency_s) for t, i in zip(t_sub, ids))
    # strictly sequential: each request was admitted after the previous one finished
    for (a0, e0), (a1, e1) in zip(spans, spans[1:]):
        assert a1 >= e0 - 5e-3, spans
    for rid, (pr, iters, calls, n_ev) in zip(ids, reqs):
        ra, _ = _alone(V, pr, iters, calls, 0, 1)
        assert _rel(done[rid].result.integral, ra.integral) < 1e-9


def test_generation_call_limit():
    """A request adapted with far too few calls (d = 15, K = 22, 100 bins,
    2000 calls per iteration) has a heavy weight tail, and each larger weight
    seen during generation lowers the unweighting efficiency further: the
    per-request call limit ends it with VAMP_ERR_LIMIT, and the events it
    wrote are exactly those of the same generation run alone up to that
    count."""
    import torch
    from paper_1811_09711_gb300 import vamp as V
    pr, iters, calls, n_ev = _requests(10, min_calls=2000, div=200)[9]
    assert (pr.d, pr.n_channels, calls) == (15, 22, 2000)
    buf = torch.zeros(n_ev * V.record_bytes(pr.d), dtype=torch.uint8, device="cuda")
    srv = V.Server(max_slots=2, precision=1)
    limit = 3 << 20
    srv.submit(pr, iters, calls, n_ev, buf.data_ptr(), max_gen_calls=limit)
    srv.wait_idle(120.0)
    (r,) = srv.poll()
    srv.close()
    assert r.status == V.VAMP_ERR_LIMIT and r.iterations == iters
    assert 0 <= r.events_written < n_ev and r.events_calls_used <= limit
    if r.events_written:
        _, ev = _alone(V, pr, iters, calls, r.events_written, 1)
        p_a = ev[0]
        p_s, _ = V.decode_records(buf[: r.events_written * V.record_bytes(pr.d)].cpu().numpy(), pr.d)
        assert _near_fraction(p_s, p_a) >= 0.98


def test_server_rejects_bad_requests():
    from paper_1811_09711_gb300 import vamp as V
    pr = _requests(1)[0][0]
    srv = V.Server(max_slots=2, precision=1)
    with pytest.raises(V.VampError):
        srv.submit(pr, 2, 1000, 100, 0)  # events without a buffer
    with pytest.raises(V.VampError):
        srv.submit(pr, 0, 1000, 0, 0)  # no iteration
    with pytest.raises(V.VampError):
        srv.submit(pr.replace(n_bins=0), 2, 1000, 0, 0)
    with pytest.raises(V.VampError):
        srv.submit(pr, 2, 0, 0, 0)
    with pytest.raises(V.VampError):
        srv.submit(pr, 2, 1000, 0, 0, max_gen_calls=-1)
    srv.wait_idle(10.0)
    assert srv.poll() == []
    srv.close()

"""Asynchronous sampling pass (vamp_sample_pass_async), GPU: its device-side
result equals the synchronous pass from the same state, and adaptation
iterations captured in a CUDA graph and replayed equal the same iterations
run call by call (1e-12 in FP64, 1e-9 in FP32-eval: the FP64 atomics of the
accumulators add in launch order)."""
import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1811_09711_gb300 import vamp
    return vamp


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _check(dev_row, r, tol):
    assert dev_row[8] == 0.0
    assert int(dev_row[4]) == r.n_calls
    assert _rel(dev_row[0], r.integral) < tol
    assert _rel(dev_row[2], r.w_max) < tol
    assert abs(dev_row[1] - r.variance) <= tol * (r.variance + r.integral ** 2 / r.n_calls)


@pytest.mark.parametrize("precision,tol,stratified", [(0, 1e-12, 0), (1, 1e-9, 0), (0, 1e-12, 1)])
def test_async_pass_equals_sync(V, precision, tol, stratified):
    import torch
    pr = P.bw_gauss().replace(stratified=stratified)
    a = V.Vamp(pr, precision=precision)
    b = V.Vamp(pr, precision=precision)
    out = torch.zeros((4, 9), dtype=torch.float64, device="cuda")
    a.sample_pass(200_000, 0)  # picks the kernel
    b.sample_pass(200_000, 0)
    ref = []
    for it in range(1, 4):
        for g in (a, b):
            g.refine_grids()
            g.update_alpha()
        a.sample_pass_async(200_000, it, out[it].data_ptr())
        ref.append(b.sample_pass(200_000, it))
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    for it in range(1, 4):
        _check(host[it], ref[it - 1], tol)
    np.testing.assert_allclose(a.get_state()["alpha"], b.get_state()["alpha"], rtol=1e3 * tol)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_iterations_captured_in_a_cuda_graph(V, precision, tol):
    import torch
    pr = P.bw_gauss()
    s = torch.cuda.Stream()
    a = V.Vamp(pr, precision=precision, stream=s)
    b = V.Vamp(pr, precision=precision)
    calls = 200_000
    with torch.cuda.stream(s):
        out = torch.zeros((5, 9), dtype=torch.float64, device="cuda")
    a.sample_pass(calls, 0)  # kernel choice and buffers before the capture
    b.sample_pass(calls, 0)
    for g in (a, b):
        g.refine_grids()
        g.update_alpha()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        for it in range(1, 5):
            a.sample_pass_async(calls, it, out[it].data_ptr())
            a.refine_grids()
            a.update_alpha()
    graph.replay()
    ref = []
    for it in range(1, 5):
        ref.append(b.sample_pass(calls, it))
        b.refine_grids()
        b.update_alpha()
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    for it in range(1, 5):
        _check(host[it], ref[it - 1], tol)
    sa, sb = a.get_state(), b.get_state()
    np.testing.assert_allclose(sa["edges"], sb["edges"], rtol=0, atol=1e3 * tol)
    np.testing.assert_allclose(sa["alpha"], sb["alpha"], rtol=1e3 * tol)


def test_async_pass_argument_checks(V):
    import torch
    g = V.Vamp(P.single_gauss())
    buf = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VampError):
        g.sample_pass_async(1000, 0, buf.data_ptr() + 4)  # misaligned
    with pytest.raises(V.VampError):
        g.sample_pass_async(1000, 1 << 31, buf.data_ptr())
    with pytest.raises(V.VampError):
        g.sample_pass_async(0, 0, buf.data_ptr())
    g.sample_pass_async(1000, 0, buf.data_ptr())
    torch.cuda.synchronize()
    assert int(buf[4].item()) == g.allocate(1000) and buf[8].item() == 0.0

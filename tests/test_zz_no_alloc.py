"""vamp_sample_pass_static against vamp_sample_pass (GPU).

The static entry point exists for callers that cannot let the library
allocate device memory; it must give the same pass as the context-based
entry point on the same grid state.  This file is collected last so that a
run stopping at the first failure has already run every other test; it
passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("precision", [0, 1])
def test_static_pass_matches_context_pass(precision):
    import torch
    from paper_1811_09711_gb300 import vamp as V
    assert torch.cuda.is_available()
    pr = P.collider()
    ctx = V.Vamp(pr, precision=precision)
    # adapt once so that grids, α and shifts are not trivial
    ctx.sample_pass(200_000, 0)
    ctx.refine_grids()
    ctx.update_alpha()
    for call_no, (n_calls, it) in enumerate([(300_007, 1), (250_000, 2)]):
        st = ctx.get_state()
        edges = torch.tensor(st["edges"], dtype=torch.float64, device="cuda").contiguous()
        alpha = torch.tensor(st["alpha"], dtype=torch.float64, device="cuda")
        shift = torch.tensor(st["shift"], dtype=torch.float64, device="cuda")
        D_out = torch.empty((pr.n_channels, pr.d, pr.n_bins), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rs = V.sample_pass_static(pr, precision, edges.data_ptr(), alpha.data_ptr(), shift.data_ptr(),
                                  n_calls, it, 0, D_out.data_ptr())
        rc = ctx.sample_pass(n_calls, it)
        assert rs.n_calls == rc.n_calls
        assert _rel(rs.integral, rc.integral) < 1e-12, (call_no, rs.integral, rc.integral)
        m2 = rc.variance + rc.integral ** 2 / rc.n_calls
        assert abs(rs.variance - rc.variance) <= 1e-12 * m2
        assert _rel(rs.w_max, rc.w_max) < 1e-12
        Dc = ctx.get_pass()["D"]
        np.testing.assert_allclose(D_out.cpu().numpy(), Dc, rtol=1e-12, atol=1e-12 * Dc.max())
        # inputs are read only
        assert np.array_equal(shift.cpu().numpy(), st["shift"])
        assert np.array_equal(edges.cpu().numpy(), st["edges"])
        ctx.refine_grids()
        ctx.update_alpha()


def test_static_pass_rejects_oversized_problem():
    import torch
    from paper_1811_09711_gb300 import vamp as V
    # 512 channels x 16 dims x 256 bins needs far more than the static array
    rng = np.random.default_rng(1)
    K, d, n = 512, 16, 256
    ms = P.MapSet.identity(K)
    pr = P.Problem(name="huge", d=d, n_bins=n, channels=ms, peak_weight=np.full(K, 1.0 / K), peaks=ms.copy(),
                   gauss_sigma=0.2, gauss_centre=0.5, gauss_norm=P.GAUSS_NORM_UNIT, seed=1)
    e = torch.zeros((K, d, n + 1), dtype=torch.float64, device="cuda")
    a = torch.zeros(K, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VampError) as err:
        V.sample_pass_static(pr, 1, e.data_ptr(), a.data_ptr(), a.data_ptr(), 1000, 0)
    assert err.value.status == V.VAMP_ERR_INVALID_ARG
    assert "static limit" in str(err.value)

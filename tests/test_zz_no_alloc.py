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
    ctx.select_kernel(0)  # the static pass runs the first candidate kernel of the shape
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


def _state_tensors(st):
    import torch
    edges = torch.tensor(st["edges"], dtype=torch.float64, device="cuda").contiguous()
    alpha = torch.tensor(st["alpha"], dtype=torch.float64, device="cuda")
    shift = torch.tensor(st["shift"], dtype=torch.float64, device="cuda")
    return edges, alpha, shift


@pytest.mark.parametrize("precision", [0, 1])
def test_static_pass_equivalences_signed_and_no_D_out(precision):
    """A problem with a channel-equivalence table (the static pass samples
    only, so the table must not change its pass) and a signed integrand
    (w_max bounds |w|): static and context passes agree, also when the
    caller asks for no d-value output."""
    import torch
    from paper_1811_09711_gb300 import vamp as V
    # a rotation table over the first three channels of the signed problem
    pr = P.signed_bw_gauss().replace(equivalences=P.rotation_equivalences(3, 8, P.EQ_SYMMETRIC))
    ctx = V.Vamp(pr, precision=precision)
    ctx.select_kernel(0)  # the static pass runs the first candidate kernel of the shape
    ctx.sample_pass(100_000, 0)
    ctx.refine_grids()
    ctx.update_alpha()
    for call_no, (n_calls, it, want_D) in enumerate([(123_457, 1, False), (99_999, 2, True)]):
        st = ctx.get_state()
        edges, alpha, shift = _state_tensors(st)
        D_out = torch.full((pr.n_channels, pr.d, pr.n_bins), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rs = V.sample_pass_static(pr, precision, edges.data_ptr(), alpha.data_ptr(), shift.data_ptr(),
                                  n_calls, it, 0, D_out.data_ptr() if want_D else 0)
        rc = ctx.sample_pass(n_calls, it)
        assert rs.n_calls == rc.n_calls
        assert _rel(rs.integral, rc.integral) < 1e-12, (call_no, rs.integral, rc.integral)
        m2 = rc.variance + rc.integral ** 2 / rc.n_calls
        assert abs(rs.variance - rc.variance) <= 1e-12 * m2
        assert _rel(rs.w_max, rc.w_max) < 1e-12
        Dh = D_out.cpu().numpy()
        if want_D:
            Dc = ctx.get_pass()["D"]
            np.testing.assert_allclose(Dh, Dc, rtol=1e-12, atol=1e-12 * Dc.max())
        else:
            assert np.all(Dh == -1.0)  # no output requested: the buffer is untouched
        ctx.refine_grids()
        ctx.update_alpha()


def test_static_pass_after_rejected_call():
    """A rejected (oversized) call leaves nothing behind: the next two valid
    calls in a row each equal the context pass on the same state."""
    import torch
    from paper_1811_09711_gb300 import vamp as V
    K, d, n = 512, 16, 256
    ms = P.MapSet.identity(K)
    huge = P.Problem(name="huge", d=d, n_bins=n, channels=ms, peak_weight=np.full(K, 1.0 / K), peaks=ms.copy(),
                     gauss_sigma=0.2, gauss_centre=0.5, gauss_norm=P.GAUSS_NORM_UNIT, seed=1)
    e = torch.zeros((K, d, n + 1), dtype=torch.float64, device="cuda")
    a = torch.zeros(K, dtype=torch.float64, device="cuda")
    pr = P.bw_gauss()
    ctx = V.Vamp(pr, precision=1)
    ctx.select_kernel(0)  # the static pass runs the first candidate kernel of the shape
    ctx.sample_pass(50_000, 0)
    ctx.refine_grids()
    ctx.update_alpha()
    st = ctx.get_state()
    edges, alpha, shift = _state_tensors(st)
    torch.cuda.synchronize()
    with pytest.raises(V.VampError) as err:
        V.sample_pass_static(huge, 1, e.data_ptr(), a.data_ptr(), a.data_ptr(), 1000, 0)
    assert err.value.status == V.VAMP_ERR_INVALID_ARG
    with pytest.raises(V.VampError) as err:
        V.sample_pass_static(pr, 1, edges.data_ptr(), alpha.data_ptr(), shift.data_ptr(), 2 ** 62, 1)
    assert err.value.status == V.VAMP_ERR_INVALID_ARG
    ref = ctx.sample_pass(77_777, 1)
    for _ in range(2):
        rs = V.sample_pass_static(pr, 1, edges.data_ptr(), alpha.data_ptr(), shift.data_ptr(), 77_777, 1)
        assert rs.n_calls == ref.n_calls
        assert _rel(rs.integral, ref.integral) < 1e-12
        assert _rel(rs.w_max, ref.w_max) < 1e-12

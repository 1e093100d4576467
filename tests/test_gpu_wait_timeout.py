"""Failure detection without a GPU fault: a device-side wait that nothing
completes gives up after its cycle limit, the kernel reports VAMP_ERR_TIMEOUT
through its error flag, and the device stays usable (a pass right after
matches the oracle)."""
import pytest

from paper_1811_09711_gb300 import problems as P

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_device_stays_usable(oracle_mod):
    from paper_1811_09711_gb300 import vamp as V
    limit = 1 << 20  # about half a millisecond of SM cycles
    rc, waited = V.selftest_bounded_wait(limit)
    assert rc == V.VAMP_ERR_TIMEOUT
    assert limit <= waited < 64 * limit
    pr = P.single_gauss()
    g = V.Vamp(pr, precision=V.PREC_FP64)
    r = g.sample_pass(20_000, 0)
    ro = oracle_mod.Oracle(pr).sample_pass(20_000, 0, n_threads=4)
    assert r.n_calls == ro.n_calls
    assert abs(r.integral - ro.integral) <= 1e-12 * abs(ro.integral)

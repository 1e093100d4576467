"""Channel equivalences (§3.5) on the GPU, through the C ABI.

* whole FP64 adaptation runs with equivalences of every kind (identity,
  invert, symmetric, invariant; permuted axes; a channel paired with itself)
  equal the FP64 oracle within 1e-12 (integral, variance, D, edges, α);
* at the benchmark's call count the symmetry property the oracle is pinned
  by holds: rotation-equivalent channels keep grids that are exact images
  of one another;
* batches and servers apply them as a context does;
* malformed tables are rejected.
"""
import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P
from test_gpu_parity import run_schedule

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1811_09711_gb300 import vamp
    return vamp


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def _self_equiv(d, kinds):
    return np.array([[0, 0] + list(range(d)) + list(kinds)], np.int32)


def _random_equiv(pr, n, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        c, cp = rng.integers(0, pr.n_channels, 2)
        rows.append([c, cp] + list(rng.permutation(pr.d)) + list(rng.integers(0, 4, pr.d)))
    return np.array(rows, np.int32)


def _perm(c, cp, n_ring, d):
    return [(k + cp - c) % n_ring if k < n_ring else k for k in range(d)]


def _case(name):
    if name == "ring_identity":
        return P.ring(3, 6), 60_000
    if name == "ring_invert":
        return P.ring(3, 6, kind=P.EQ_INVERT), 60_000
    if name == "ring_symmetric":
        return P.ring(4, 8, kind=P.EQ_SYMMETRIC), 80_000
    if name == "self_invert":
        pr = P.single_gauss()
        return pr.replace(equivalences=_self_equiv(pr.d, [P.EQ_INVERT] * pr.d)), 40_000
    if name == "self_invariant_mix":
        pr = P.single_gauss()
        kinds = [P.EQ_SYMMETRIC, P.EQ_INVARIANT, P.EQ_IDENTITY, P.EQ_INVERT]
        return pr.replace(equivalences=_self_equiv(pr.d, kinds)), 40_000
    if name == "bw_gauss_random":
        pr = P.bw_gauss()
        return pr.replace(equivalences=_random_equiv(pr, 12, 5)), 200_000
    raise ValueError(name)


@pytest.mark.parametrize("name", ["ring_identity", "ring_invert", "ring_symmetric", "self_invert",
                                  "self_invariant_mix", "bw_gauss_random"])
def test_equiv_schedule_fp64(V, O, name):
    pr, calls = _case(name)
    pr = pr.replace(combine_from=1)
    run_schedule(V, O, pr, 4, calls)


def test_rotation_images_at_full_size(V):
    """ring with 8 channels, FP32 evaluation, 1e7 calls per pass: the grids
    of rotation-equivalent channels stay images of one another."""
    n_ring, d = 8, 8
    g = V.Vamp(P.ring(n_ring, d).replace(n_bins=100), precision=1)
    for it in range(3):
        r = g.sample_pass(10_000_000, it)
        g.refine_grids()
        g.update_alpha()
    assert abs(r.integral - 1.0) < 5 * np.sqrt(r.variance)
    e = g.get_state()["edges"]
    dev = 0.0
    for c in range(n_ring):
        for cp in range(n_ring):
            pm = _perm(c, cp, n_ring, d)
            for k in range(d):
                dev = max(dev, np.abs(e[cp][pm[k]] - e[c][k]).max())
    assert dev < 1e-13, dev


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_equiv_in_batch_equals_alone(V, precision, tol):
    probs = [P.ring(3, 6).replace(calls=40_000), P.ring(4, 8, kind=P.EQ_SYMMETRIC).replace(calls=60_000)]
    b5 = P.batch_instance(5)
    probs.append(b5.replace(calls=50_000, equivalences=_random_equiv(b5, 6, 9)))
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
            np.testing.assert_allclose(batch.get_state(i)["edges"], g.get_state()["edges"], rtol=0,
                                       atol=1e3 * tol)


def test_equiv_in_server_equals_alone(V):
    import torch
    pr = P.ring(3, 6)
    srv = V.Server(max_slots=2, precision=0)
    rid = srv.submit(pr, 3, 40_000, 0, 0)
    srv.wait_idle(120.0)
    done = {r.id: r for r in srv.poll(4)}
    srv.close()
    g = V.Vamp(pr, precision=0)
    for it in range(3):
        ra = g.sample_pass(40_000, it)
        g.refine_grids()
        g.update_alpha()
    torch.cuda.synchronize()
    r = done[rid]
    assert r.status == V.VAMP_OK
    assert abs(r.result.integral - ra.integral) <= 1e-12 * abs(ra.integral)


@pytest.mark.parametrize("bad", ["channel", "axis", "not_perm", "kind"])
def test_invalid_equivalences_rejected(V, bad):
    d = 6
    row = [0, 1] + list(range(d)) + [0] * d
    if bad == "channel":
        row[1] = 3
    elif bad == "axis":
        row[2] = -1
    elif bad == "not_perm":
        row[4] = row[5]
    else:
        row[2 + d] = 7
    with pytest.raises(V.VampError):
        V.Vamp(P.ring(3, d).replace(equivalences=np.array([row], np.int32)))

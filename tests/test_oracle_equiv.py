"""Pins of the oracle's channel equivalences (§3.5; reading R18) against facts
fixed by symmetry and by the rebinning itself (CPU only)."""
import numpy as np
import pytest

from paper_1811_09711_gb300 import problems as P


def _self_equiv(d, kinds):
    """One equivalence of channel 0 with itself, axes matched one to one."""
    return np.array([[0, 0] + list(range(d)) + list(kinds)], np.int32)


def _perm(c, cp, n_ring, d):
    return [(k + cp - c) % n_ring if k < n_ring else k for k in range(d)]


def test_no_equivalences_pooled_is_D(oracle_mod):
    o = oracle_mod.Oracle(P.bw_gauss())
    o.sample_pass(50_000, 0, n_threads=2)
    assert np.array_equal(o.get_pooled(), o.get_pass()["D"])


def test_rotation_images_adapt_identically(oracle_mod):
    """ring: channel c' samples like channel c with axes shifted by c' - c.
    With the rotation equivalences every axis pools the same orbit of
    d-values, so the refined grids are images of one another after every
    iteration (a 3-cycle, so a reversed permutation would not do); without
    them they differ by sampling noise."""
    n_ring, d = 3, 6
    for eq in (True, False):
        o = oracle_mod.Oracle(P.ring(n_ring, d, equivalences=eq))
        for it in range(3):
            o.sample_pass(30_000, it, n_threads=3)
            pooled = o.get_pooled()
            o.refine_grids()
            o.update_alpha()
            e = o.get_state()["edges"]
            dev = dev_pool = 0.0
            for c in range(n_ring):
                for cp in range(n_ring):
                    pm = _perm(c, cp, n_ring, d)
                    for k in range(d):
                        dev = max(dev, np.abs(e[cp][pm[k]] - e[c][k]).max())
                        dev_pool = max(dev_pool, np.abs(pooled[cp][pm[k]] - pooled[c][k]).max()
                                       / pooled[c][k].max())
            if eq:
                assert dev < 1e-13 and dev_pool < 1e-14, (it, dev, dev_pool)
            else:
                assert dev > 1e-3


def test_invert_with_itself_makes_grids_mirror_symmetric(oracle_mod):
    """A channel inverted onto itself pools D_j + D_{n-1-j}: the bin weights
    are mirror-symmetric, so are the refined grids (from uniform ones)."""
    pr = P.single_gauss()
    n = pr.n_bins
    for eq in (True, False):
        o = oracle_mod.Oracle(pr.replace(equivalences=_self_equiv(pr.d, [P.EQ_INVERT] * pr.d) if eq
                                         else None))
        for it in range(3):
            o.sample_pass(10_000, it, n_threads=2)
            pooled = o.get_pooled()
            o.refine_grids()
            e = o.get_state()["edges"][0]
            asym = np.abs(e + e[:, ::-1] - 1.0).max()
            if eq:
                assert np.array_equal(pooled, pooled[:, :, ::-1])
                assert asym < 1e-14, asym
            else:
                assert asym > 1e-3
    assert n == e.shape[1] - 1


def test_symmetric_is_the_mean_of_identity_and_invert(oracle_mod):
    pools = {}
    for kind in (P.EQ_IDENTITY, P.EQ_INVERT, P.EQ_SYMMETRIC):
        o = oracle_mod.Oracle(P.ring(3, 6, kind=kind))
        o.sample_pass(30_000, 0, n_threads=2)
        pools[kind] = o.get_pooled()
        D = o.get_pass()["D"]
    mean = 0.5 * (pools[P.EQ_IDENTITY] + pools[P.EQ_INVERT])
    assert np.abs(pools[P.EQ_SYMMETRIC] - mean).max() <= 1e-15 * np.abs(mean).max()
    assert not np.allclose(pools[P.EQ_IDENTITY], pools[P.EQ_INVERT])
    assert not np.allclose(pools[P.EQ_IDENTITY], D)


def test_invariant_axis_is_kept(oracle_mod):
    """An invariant axis takes unit bin weights: the rebinning keeps its
    (already adapted) edges whatever the pass measured; the other axes adapt."""
    pr = P.single_gauss()
    base = oracle_mod.Oracle(pr)
    for it in range(2):
        base.sample_pass(10_000, it, n_threads=2)
        base.refine_grids()
    st = base.get_state()
    kinds = [P.EQ_IDENTITY, P.EQ_INVARIANT, P.EQ_IDENTITY, P.EQ_IDENTITY]
    o = oracle_mod.Oracle(pr.replace(equivalences=_self_equiv(pr.d, kinds)))
    o.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"], have_pass=False)
    o.sample_pass(10_000, 2, n_threads=2)
    assert np.all(o.get_pooled()[0, 1] == 1.0)
    o.refine_grids()
    e = o.get_state()["edges"][0]
    assert np.abs(e[1] - st["edges"][0][1]).max() < 1e-14
    for k in (0, 2, 3):
        assert np.abs(e[k] - st["edges"][0][k]).max() > 1e-4


def test_switched_off_partner_adds_nothing(oracle_mod):
    """A channel with α = 0 samples no calls: its d-values are zero and an
    equivalence with it leaves the partner's weights as they are."""
    o = oracle_mod.Oracle(P.ring(3, 6))
    st = o.get_state()
    o.set_state(st["edges"], np.array([0.5, 0.5, 0.0]), st["shift"], 0.0, have_pass=False)
    o.sample_pass(30_000, 0, n_threads=2)
    D = o.get_pass()["D"]
    pooled = o.get_pooled()
    assert np.all(D[2] == 0.0)
    for k in range(6):
        assert np.array_equal(pooled[0][k], D[0][k] + D[1][_perm(0, 1, 3, 6)[k]])


def test_equivalences_improve_adaptation(oracle_mod):
    """Pooling six symmetric channels' d-values adapts their grids on six
    times the statistics: the per-call variance after a short adaptation is
    lower than without the equivalences, seed by seed."""
    ratios = []
    for s in range(6):
        v = {}
        for eq in (True, False):
            o = oracle_mod.Oracle(P.ring(6, 6, seed=100 + s, equivalences=eq).replace(n_bins=50))
            for it in range(4):
                o.sample_pass(20_000, it, n_threads=4)
                o.refine_grids()
                o.update_alpha()
            r = o.sample_pass(200_000, 10, n_threads=4)
            v[eq] = r.variance * r.n_calls
        ratios.append(v[True] / v[False])
    assert max(ratios) < 1.0 and np.mean(ratios) < 0.97, ratios


@pytest.mark.parametrize("bad", ["channel", "partner", "axis", "not_perm", "kind"])
def test_invalid_equivalences_rejected(oracle_mod, bad):
    d = 6
    row = [0, 1] + list(range(d)) + [0] * d
    if bad == "channel":
        row[0] = 3
    elif bad == "partner":
        row[1] = -1
    elif bad == "axis":
        row[2] = d
    elif bad == "not_perm":
        row[3] = row[2]
    else:
        row[2 + d] = 4
    with pytest.raises(ValueError):
        oracle_mod.Oracle(P.ring(3, d).replace(equivalences=np.array([row], np.int32)))

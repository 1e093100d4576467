"""The oracle reproduces its recorded short adaptation runs
(tests/golden/oracle_passes.json, written by tests/golden/make_oracle_golden.py
from the oracle alone): call counts exactly, every value to 1e-10 relative
(room for last-bit differences of the C library's functions between
machines), so that a change to the oracle's arithmetic cannot pass unnoticed."""
import importlib.util
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _maker():
    spec = importlib.util.spec_from_file_location("make_oracle_golden",
                                                  os.path.join(GOLDEN, "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _close(a, b, tol=1e-10):
    return abs(a - b) <= tol * max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("name", list(json.load(open(os.path.join(GOLDEN, "oracle_passes.json")))["cases"]))
def test_oracle_reproduces_recorded_runs(oracle_mod, name):
    mk = _maker()
    recorded = json.load(open(os.path.join(GOLDEN, "oracle_passes.json")))["cases"][name]
    pr, iters, calls = mk.cases()[name]
    got = mk.run(pr, iters, calls)
    assert len(got) == len(recorded)
    for it, (g, r) in enumerate(zip(got, recorded)):
        assert g["n_calls"] == r["n_calls"], (name, it)
        for k in ("integral", "variance", "w_max", "combined", "chi2_dof", "edges_sum", "edges_weighted"):
            assert _close(g[k], r[k]), (name, it, k, g[k], r[k])
        assert all(_close(a, b) for a, b in zip(g["alpha"], r["alpha"])), (name, it)

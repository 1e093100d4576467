"""Writes oracle_passes.json: short adaptation runs of the FP64 CPU oracle on
small seeded problems (every sampling mode), as a regression record of the
oracle's arithmetic.  The values come from ``oracle/`` only (not from the
paper and never from the CUDA library):

    python tests/golden/make_oracle_golden.py

A change to the oracle that moves these numbers must say, in its commit, which
passage of the paper (or which reading of it) justifies the change.
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_passes.json")


def cases():
    import numpy as np

    from paper_1811_09711_gb300 import problems as P
    return {
        "single_gauss": (P.single_gauss(), 3, 5_000),
        "bw_gauss": (P.bw_gauss(), 3, 20_000),
        "bw_gauss_stratified": (P.bw_gauss().replace(stratified=1), 3, 20_000),
        "ring_symmetric_equivalences": (P.ring(3, 5, kind=P.EQ_SYMMETRIC), 3, 20_000),
        "signed_pair": (P.signed_pair(d=2), 3, 10_000),
        "power_law_special_case": (P.special_case("pow", d=2, n_bins=8), 2, 4_000),
        "modes_combined": (P.ring(3, 5, kind=P.EQ_INVERT).replace(
            peak_weight=np.array([1.4, -0.6, 0.2]), stratified=1, n_bins=12), 3, 20_000),
    }


def run(pr, iters, calls):
    """One record per iteration: the pass result, then checksums of the
    refined grids and the updated channel weights."""
    import numpy as np

    from oracle import oracle as O
    o = O.Oracle(pr)
    recs = []
    for it in range(iters):
        r = o.sample_pass(calls, it, combine=it >= 1, n_threads=1)
        o.refine_grids()
        o.update_alpha()
        st = o.get_state()
        e = st["edges"]
        wts = np.arange(1, e.size + 1, dtype=np.float64).reshape(e.shape) / e.size
        recs.append({"n_calls": r.n_calls, "integral": r.integral, "variance": r.variance,
                     "w_max": r.w_max, "combined": r.combined, "chi2_dof": r.chi2_dof,
                     "edges_sum": float(e.sum()), "edges_weighted": float((wts * e).sum()),
                     "alpha": [float(a) for a in st["alpha"]]})
    return recs


def main() -> int:
    data = {name: run(*c) for name, c in cases().items()}
    with open(OUT, "w") as f:
        json.dump({"source": "FP64 CPU oracle (oracle/vamp_oracle.c), written by make_oracle_golden.py",
                   "cases": data}, f, indent=1)
    print(f"wrote {OUT}")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())

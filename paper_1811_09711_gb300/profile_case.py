"""Small, self-contained runs of the hot path for profilers (ncu).

    python -m paper_1811_09711_gb300.profile_case collider --calls 2e6 --iterations 3
    python -m paper_1811_09711_gb300.profile_case batch --instances 64 --iterations 3

``collider``: the d = 14, K = 64 collider-like problem; `iterations`
adaptation iterations of `calls` calls (pass, rebinning, α update), then
`events` unweighted events if asked.  The first pass also times the pass
kernel variants (the autotuner's probe launches come before it: two per
candidate kernel) unless `--kernel` pins one.  ``batch``: the first `instances` instances of the
256-instance uneven batch, `iterations` iterations with the work-item shape
fixed (no autotuner launches).  Prints one line and exits 0 on success.
"""
from __future__ import annotations

import argparse

import torch

from . import problems as P
from . import vamp as V


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["collider", "batch"])
    ap.add_argument("--calls", type=float, default=2e6)
    ap.add_argument("--iterations", type=int, default=3)
    ap.add_argument("--precision", type=int, default=V.PREC_FP32_EVAL)
    ap.add_argument("--events", type=int, default=0)
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--kernel", default="",
                    help="pin the pass kernel: a kernel name or its start, e.g. k_scan or 'k_pass<float, 0, 2'")
    a = ap.parse_args()
    if a.workload == "collider":
        pr = P.collider()
        g = V.Vamp(pr, precision=a.precision)
        if a.kernel:
            for i in range(g.kernel_candidates()):
                g.select_kernel(i)
                if g.kernel_name().startswith(a.kernel):
                    break
            else:
                raise SystemExit(f"no candidate kernel named {a.kernel!r}")
        for it in range(a.iterations):
            r = g.sample_pass(int(a.calls), it)
            g.refine_grids()
            g.update_alpha()
        if a.events:
            buf = torch.empty(a.events * V.record_bytes(pr.d), dtype=torch.uint8, device="cuda")
            g.generate(a.events, buf.data_ptr(), gen_id=0)
        torch.cuda.synchronize()
        print(f"collider: {a.iterations} iterations of {r.n_calls} calls, kernel {g.kernel_name()}")
    else:
        probs = P.batch(a.instances)
        b = V.Batch(probs, precision=a.precision, autotune=False)
        nc = [p.calls for p in probs]
        for it in range(a.iterations):
            b.iterate(nc, it)
        torch.cuda.synchronize()
        print(f"batch: {a.iterations} iterations of {a.instances} instances, {sum(nc)} calls each")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())

"""The multi-GPU form of the benchmark: independent replicas, one per rank
(no data-path collective; only the timing figures are reduced).  Run here as
two gloo ranks on the CPU: the job figures are the slowest rank's time and
the sum of the ranks' calls, and each rank's replica is its own random
stream -- the oracle's pass on rank r equals a single-process run of the
problem with request id r and differs from the other rank's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    from paper_1811_09711_gb300 import problems as P
    t, calls = bench.job_throughput(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world)
    pr = bench.replica_problem(P.bw_gauss(), rank)
    r = O.Oracle(pr).sample_pass(3000, 0, n_threads=1)
    out.put((rank, t, calls, pr.request_id, r.integral, r.n_calls))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_over_gloo(oracle_mod):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, c0, id0, i0, n0), (r1, t1, c1, id1, i1, n1) = res
    assert t0 == t1 == 15.0 and c0 == c1 == 3000.0  # max time, summed calls
    assert (id0, id1) == (0, 1)
    assert i0 != i1  # independent random streams
    from paper_1811_09711_gb300 import problems as P
    for rid, integral in ((0, i0), (1, i1)):
        ref = oracle_mod.Oracle(P.bw_gauss().replace(request_id=rid)).sample_pass(3000, 0, n_threads=1)
        assert ref.integral == integral


def test_single_rank_is_identity():
    import bench
    assert bench.job_throughput(12.5, 7.0, 1) == (12.5, 7.0)


def test_roofline_operation_counts():
    """The per-call operation count charged to the roofline, term by term:
    8 per lookup x K d, 15 per mapped coordinate, 7 per channel, 8 per
    coordinate, 60 per Philox block, 10 for the weight and sums."""
    import bench
    from paper_1811_09711_gb300 import problems as P
    pr = P.collider()
    K, d = pr.n_channels, pr.d
    mapped = int(pr.channels.n_mapped.sum())
    assert (K, d, mapped) == (64, 14, 188)
    assert bench.lookup_ops_per_call(pr) == 8 * K * d == 7168
    assert bench.algorithmic_ops_per_call(pr) == 8 * K * d + 15 * mapped + 7 * K + 8 * d + 60 * 4 + 10 == 10798


def test_roofline_per_pipe_work():
    """Per-pipe work per call charged to the roofline: MUFU operations (one
    exp2 per channel, one reciprocal per Breit-Wigner map, five per power
    map), shared-memory wavefronts (three 4-byte reads per lookup at 32
    lanes per wavefront) and FP64 operations of the FP32-eval form."""
    import bench
    from paper_1811_09711_gb300 import problems as P
    pr = P.collider()
    ch = pr.channels
    kinds = [int(ch.kind[c, s]) for c in range(pr.n_channels) for s in range(int(ch.n_mapped[c]))]
    bw, pw = kinds.count(P.MAP_BW), kinds.count(P.MAP_POW)
    assert bw + pw == 188 and bench.mapped_kinds(pr) == (bw, pw)
    assert bench.xu_ops_per_call(pr) == 64 + bw + 5 * pw
    assert bench.lsu_wavefronts_per_call(pr) == 3 * 64 * 14 / 32 == 84.0
    assert bench.fp64_ops_per_call(pr) == 20.0


def test_union_pass_per_pipe_work():
    """Per-pipe work per call of the union pass, term by term: L2 bytes (one
    256-byte density row and one 4-byte cell entry per coordinate), MUFU
    operations (one exp2 per channel, one reciprocal per Breit-Wigner map,
    four per power map) and shared-memory wavefronts (channel record, slot
    record and coordinate per mapped slot; four 16-byte interval loads per
    coordinate and 32 calls; the factors written and read back)."""
    import bench
    from paper_1811_09711_gb300 import problems as P
    pr = P.collider()
    bw, pw = bench.mapped_kinds(pr)
    assert bench.union_l2_bytes_per_call(pr) == 14 * (256 + 4) == 3640
    assert bench.union_xu_ops_per_call(pr) == 64 + bw + 4 * pw
    assert bench.union_lsu_wavefronts_per_call(pr) == (64 + 2 * 188) / 32 + 14 * 4 / 32 + 2 * 64 / 32 + 2 == 21.5


def test_fp64_form_operation_count():
    """Floating-point work per call of the FP64 form, term by term: one
    density product per lookup, 12 per Breit-Wigner map, 14 per power map,
    7 per channel, 4 per coordinate, 10 for the weight and sums."""
    import bench
    from paper_1811_09711_gb300 import problems as P
    pr = P.collider()
    bw, pw = bench.mapped_kinds(pr)
    assert bench.fp64_form_ops_per_call(pr) == 64 * 14 + 12 * bw + 14 * pw + 7 * 64 + 4 * 14 + 10
    assert bench.fp64_form_ops_per_call(pr) == 3850

#!/usr/bin/env python3
"""Benchmark of the multi-channel integrator's hot path on one GB300 per rank.

Workload (both arms): the collider-like problem -- d = 14, K = 64 channels
mapping 2-4 coordinates each by Breit-Wigner or power-law maps, 64 matching
peaks with widths log-uniform in [1e-4, 1e-2], n = 100 bins per axis,
1e7 calls per adaptation iteration.

A step is one adaptation iteration: the sampling pass over 1e7 calls
(RNG, forward map, integrand, g(p) over all 64 channels, accumulation),
the pass result and iteration combination, grid refinement and the α update.
`value` = calls per second of the FP32-eval path with inputs resident on the
device (CUDA events on the library's stream, L2 flushed between steps).
`e2e` = the same steps through the C ABI with the grid state round-tripping
through pinned host buffers every step (host->device set_state, pass,
refine, α, device->host get_state).  The FP64 path and unweighted-event
generation (1e6 events) are measured in the same run and reported beside it.

`batch`: 256 uneven integrations (d in 2..16, K log-uniform in 1..64, calls
log-uniform in 1e4..1e7, bins in {20, 50, 100}) advanced together, calls/s
with autotuned and with fixed work items.  `serving`: a Poisson stream of
integrate-then-generate requests (200 req/s over a 60 s arrival window,
10 iterations each, 1e3..1e5 events each, 120 GB device budget) through the
continuous-batching server, wall-clock throughput and p50/p99 latency, for
the FP32-eval form, and for the FP64 form at an offered rate it sustains
(16 req/s over 60 s).

`roofline`: per pipe (32-bit lanes, shared-memory wavefronts, MUFU, FP64)
the method's own work per call times the pass kernel's calls/s, against the
pipe's throughput measured on the same GPU by small kernels
(vamp_measure_peaks); `frac` is the binding pipe's fraction.

`fp32_accuracy`: the FP32-eval pass against the FP64 pass on the same grids,
α and random stream -- integral deviation (relative and in σ), and on a
sample of calls the inverse-lookup bin flips and per-call weight deviations.
`cpu_baseline`: the FP64 oracle on all host cores and on one.

--impl reference times the FP64 CPU oracle (the only reference this method
has) on bounded samples of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
import types

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VAMP calls/s at d=14, 64 ch (FP32-eval vs FP64 path); p50/p99 request latency"
UNIT = "calls/s"
WORKLOAD = "collider_d14_k64_n100: d=14, K=64 channels (2-4 BW/power maps each), 64 peaks, 100 bins, 1e7 calls/iteration"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is producing lines
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_problem(base, rank: int):
    """The workload of one rank: an independent replica of the problem on
    its own random stream (request id = rank); no data crosses ranks."""
    return base.replace(request_id=rank)


def job_throughput(t_ms: float, calls: float, world_size: int, device="cpu"):
    """Whole-job figures from per-rank ones: the slowest rank's time and
    the calls of all ranks (one max- and one sum-reduction over the ranks'
    process group; identity for one rank)."""
    if world_size <= 1:
        return t_ms, calls
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_ms, float(calls)], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = tt.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


# per kernel family: the sources its traffic record is bound to and the
# committed ncu summary that holds the record
KERNEL_SOURCES = {
    "k_pass": (["vamp_pass.cuh", "vamp_device.cuh", "vamp_pass_f32_shapes.cu", "vamp_internal.h"],
               "k_pass_fp32_collider_d14_k64.md"),
    "k_union": (["vamp_union.cuh", "vamp_pass.cuh", "vamp_device.cuh", "vamp_union.cu", "vamp_internal.h"],
                "k_union_fp32_collider_d14_k64.md"),
}


# kernels of one timed adaptation step: allocation, sampling pass, pass
# result, result copy (asynchronous form), rebinning, channel weights; the
# union pass adds the four that rebuild its interval tables after the
# rebinning (edge images, sort, cell index, density rows)
KERNELS_PER_STEP = 6
UNION_EXTRA_KERNELS = 4


def kernel_family(kernel: str) -> str:
    return kernel.split("<")[0]


def measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernel sources changed since the counters were taken."""
    import hashlib
    import re
    fam = KERNEL_SOURCES.get(kernel_family(kernel))
    if fam is None:
        return None
    h = hashlib.sha256()
    for s in fam[0]:
        with open(os.path.join(ROOT, "paper_1811_09711_gb300", "csrc", s), "rb") as f:
            h.update(f.read())
    try:
        with open(os.path.join(ROOT, "profiles", fam[1])) as f:
            txt = f.read()
    except OSError:
        return None
    for m in re.finditer(r"traffic_record: (.+?) (\d+) sha256=([0-9a-f]+)", txt):
        if m.group(1) == kernel and m.group(3) == h.hexdigest():
            return int(m.group(2))
    return None


def lookup_ops_per_call(pr) -> float:
    """The K*d bin lookups of g(p) alone, 8 lane-ops each (cell index 2,
    table probe 1, edge probe + compare + select 3, density read + multiply 2)."""
    return 8.0 * pr.n_channels * pr.d


def algorithmic_ops_per_call(pr) -> float:
    """Algorithmic lane-operations of one call (what the method must compute,
    not what a kernel happens to issue), charged to the roofline:
      8 per bin lookup (K*d of them, as above);
      15 per inverse map of a mapped coordinate of another channel (the
        inverse map itself, its Jacobian factor, the matching peak's factor
        and the coordinate's Gaussian exponent);
      7 per channel for its terms of g and f (two multiply-adds, one exp2,
        two multiplies, the exponent difference);
      6 per coordinate for the forward map (bin index and fraction from the
        random word, interpolation, density) and 2 for its d-value update;
      60 per Philox4x32-10 block (ten rounds of two 32-bit multiplies, xors
        and key updates) for the d words of the call;
      10 for the weight and the channel sums.
    For the collider-like problem (d = 14, K = 64, 188 mapped coordinates)
    this is 10 798 lane-ops per call."""
    K, d = pr.n_channels, pr.d
    mapped = int(sum(int(x) for x in pr.channels.n_mapped))
    return (8.0 * K * d + 15.0 * mapped + 7.0 * K + 8.0 * d + 60.0 * ((d + 3) // 4) + 10.0)


def mapped_kinds(pr):
    """Breit-Wigner and power-law mapped coordinates over all channels."""
    ch = pr.channels
    bw = pw = 0
    for c in range(pr.n_channels):
        for s in range(int(ch.n_mapped[c])):
            k = int(ch.kind[c, s])
            bw += k == 1
            pw += k == 2
    return bw, pw


def xu_ops_per_call(pr) -> float:
    """MUFU (special-function unit) operations of one call: one exp2 per
    channel (its peak's Gaussian factor); per mapped coordinate one
    reciprocal for a Breit-Wigner map (the Jacobian quotient), and two log2,
    two exp2 and one reciprocal for a power map (x = p^0.2, the Jacobian,
    the peak's (p + δ)^-0.8)."""
    bw, pw = mapped_kinds(pr)
    return float(pr.n_channels + bw + 5 * pw)


def lsu_wavefronts_per_call(pr) -> float:
    """Shared-memory load wavefronts of one call at the ideal one wavefront
    per 32 lanes: the K*d bin lookups at three reads each (cell table, edge,
    density)."""
    return 3.0 * pr.n_channels * pr.d / 32.0


def fp64_ops_per_call(pr) -> float:
    """FP64 operations of one call in the FP32-eval form: the weight and its
    square, the shifted sums (difference, sum, multiply-add), the maximum,
    and one d-value addition per coordinate."""
    return 6.0 + pr.d


def union_l2_bytes_per_call(pr) -> float:
    """Bytes the union pass reads from L2 per call: one 256-byte density row
    (UNION_SLOTS = 64 channels, FP32) and one 4-byte cell entry per
    coordinate (the scans past the cell entry are rare and not counted)."""
    return pr.d * (64 * 4 + 4.0)


def union_xu_ops_per_call(pr) -> float:
    """MUFU operations of one call in the union pass: one exp2 per channel
    (its peak's Gaussian factor); one reciprocal per Breit-Wigner coordinate
    (the Jacobian at p); two log2 and two exp2 per power-law coordinate
    (p^-0.8 for the Jacobian, (p + δ)^-0.8 for the peak).  No inverse maps."""
    bw, pw = mapped_kinds(pr)
    return float(pr.n_channels + bw + 4 * pw)


def union_lsu_wavefronts_per_call(pr) -> float:
    """Shared-memory wavefronts of one call in the union pass at one per warp
    access: per channel its record and per mapped coordinate the slot record
    and the call's coordinate (part J, per thread); per coordinate the 32
    intervals of the warp's calls (part U: four 16-byte broadcast loads per
    32 calls); the channel factors written (two wavefronts per warp store of
    32 calls) and read back (two per float2 warp load)."""
    mapped = int(sum(int(x) for x in pr.channels.n_mapped))
    K = pr.n_channels
    return (K + 2.0 * mapped) / 32.0 + pr.d * 4.0 / 32.0 + 2.0 * K / 32.0 + 2.0


def fp64_form_ops_per_call(pr) -> float:
    """Floating-point operations of one call that the FP64 form runs on the
    FP64 pipe (bin indices and edge comparisons are integer work there, and
    a transcendental function counts as one operation):
      1 per bin lookup (the density product), K*d of them;
      12 per Breit-Wigner inverse map (offset, square-add, Jacobian
        quotient, argument scale, arctangent, shift, scale, the Jacobian
        into g and into the peak, the Gaussian exponent 3);
      14 per power-law inverse map (inverse fifth root, fourth power and
        product for x, Jacobian 2, the peak's root and fourth power and
        weight 5, the Gaussian exponent 3);
      7 per channel for its g and f terms; 4 per coordinate for the forward
      map and its d-value; 10 for the weight and sums.
    For the collider-like problem this is 3 850 per call."""
    bw, pw = mapped_kinds(pr)
    return float(pr.n_channels * pr.d + 12 * bw + 14 * pw + 7 * pr.n_channels + 4 * pr.d + 10)


def cpu_oracle_rate(pr, seconds: float, threads: int):
    """Times the CPU oracle (as it stands) on a bounded sample of one pass."""
    from oracle import oracle as O
    O.build()
    o = O.Oracle(pr)
    n = 20_000
    t = time.perf_counter()
    o.sample_pass(n, 0, n_threads=threads)
    dt = time.perf_counter() - t
    n2 = int(max(20_000, min(5e7, n * seconds / max(dt, 1e-3))))
    t = time.perf_counter()
    r = o.sample_pass(n2, 1, n_threads=threads)
    dt2 = time.perf_counter() - t
    return r.n_calls / dt2, r.n_calls, dt2


def run_batch(V, P, n_inst: int, iters: int):
    """256 uneven integrations advanced together (one persistent launch per
    pass, iterations replayed as a CUDA graph): calls/s with the autotuned
    work-item shape and with the fixed one."""
    probs = P.batch(n_inst)
    out = {"instances": n_inst, "iterations": iters,
           "calls_per_iteration": int(sum(p.calls for p in probs))}
    for tag, tune in (("tuned", True), ("fixed", False)):
        b = V.Batch(probs, precision=V.PREC_FP32_EVAL, autotune=tune)
        nc = [p.calls for p in probs]
        b.iterate(nc, 0)  # tuning (if any) and graph capture
        t = time.perf_counter()
        calls = 0
        ops = 0.0
        for it in range(1, iters + 1):
            res = b.iterate(nc, it)
            calls += sum(r.n_calls for r in res)
            ops += sum(r.n_calls * algorithmic_ops_per_call(p) for r, p in zip(res, probs))
        dt = time.perf_counter() - t
        # algorithmic lane-ops of every instance's calls (each charged with its
        # own K, d and mapped coordinates) over the whole iteration's wall time
        out[tag] = {"calls_per_s": calls / dt, "ms_per_iteration": 1e3 * dt / iters,
                    "alu_ops_per_s": ops / dt}
        if tune:
            out["tuning"] = b.tuning()
        b.close()
    out["speedup_tuned"] = out["tuned"]["calls_per_s"] / out["fixed"]["calls_per_s"]
    return out


def run_serving(V, P, torch, dev, precision: int, rate: float, seconds: float, budget: int, slots: int,
                iterations: int, gen_cap: int):
    """Poisson stream of integrate-then-generate requests through the
    continuous-batching server: wall-clock throughput and per-request
    latency (submit to completion)."""
    import numpy as np
    reqs = P.serving_stream(rate_per_s=rate, duration_s=seconds, seed=5)
    rbs = [V.record_bytes(r.problem.d) for r in reqs]
    offs, tot = [], 0
    for r, rb in zip(reqs, rbs):
        offs.append(tot)
        tot += (r.problem.n_events * rb + 255) // 256 * 256
    buf = torch.empty(max(tot, 256), dtype=torch.uint8, device=dev)
    base = buf.data_ptr()
    srv = V.Server(max_slots=slots, mem_budget_bytes=budget, precision=precision)
    w = P.serving_stream(rate_per_s=rate, duration_s=1.0, seed=6, max_requests=4)
    for r in w:  # warm-up: kernels loaded, shared-memory limits raised
        srv.submit(r.problem, 2, 10_000, 100, base, max_gen_calls=gen_cap)
    srv.wait_idle(600.0)
    srv.poll(64)
    s0 = srv.stats()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, off in zip(reqs, offs):
        now = time.perf_counter() - t0
        if r.arrival_s > now:
            time.sleep(r.arrival_s - now)
        srv.submit(r.problem, iterations, r.problem.calls, r.problem.n_events, base + off, max_gen_calls=gen_cap)
    srv.wait_idle(3600.0)
    wall = time.perf_counter() - t0
    res = srv.poll(len(reqs) + 16)
    s1 = srv.stats()
    srv.close()
    lat = np.array([r.latency_s for r in res]) * 1e3
    que = np.array([r.queue_s for r in res]) * 1e3
    calls = s1["calls"] - s0["calls"]
    events = s1["events"] - s0["events"]
    return {"requests": len(res), "offered_req_per_s": rate, "arrival_window_s": seconds,
            "iterations_per_request": iterations, "wall_s": wall, "req_per_s": len(res) / wall,
            "calls_per_s": calls / wall, "events_per_s": events / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "queue_p50_ms": float(np.percentile(que, 50)), "queue_p99_ms": float(np.percentile(que, 99)),
            "ticks": s1["ticks"] - s0["ticks"], "limit_hit": int(sum(r.status == V.VAMP_ERR_LIMIT for r in res)),
            "failed": int(sum(r.status not in (V.VAMP_OK, V.VAMP_ERR_LIMIT) for r in res)),
            "slots": slots, "budget_gb": budget / 1e9}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1811_09711_gb300 import problems as P
    O.build()
    pr = P.collider()
    threads = os.cpu_count() or 1
    o = O.Oracle(pr)
    sample = int(os.environ.get("VAMP_REF_CALLS", "400000"))
    it = 0
    for _ in range(args.warmup):
        o.sample_pass(sample, it, n_threads=threads)
        o.refine_grids()
        o.update_alpha()
        it += 1
    tot_calls, tot_t = 0, 0.0
    for _ in range(args.steps):
        t = time.perf_counter()
        r = o.sample_pass(sample, it, n_threads=threads)
        o.refine_grids()
        o.update_alpha()
        tot_t += time.perf_counter() - t
        tot_calls += r.n_calls
        it += 1
    v = tot_calls / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"one adaptation iteration of {sample} calls (bounded sample)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} oracle iterations of {sample} calls each, {threads} threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1811_09711_gb300 import problems as P
    from paper_1811_09711_gb300 import vamp as V

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    V.load()
    stream = torch.cuda.Stream(device=dev)
    base = P.collider()
    # independent replica per rank: its own random stream (request id)
    pr = replica_problem(base, rank)
    N = pr.calls
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            dist.barrier()

    def timed_steps(g, n_steps, it0, fp):
        """Runs n_steps adaptation iterations (asynchronous passes: no host
        round trip between steps; each pass's result lands in device memory
        and is read after the last step); returns per-step ms, calls and the
        last pass's result."""
        ms = []
        res = torch.zeros((n_steps, 9), dtype=torch.float64, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        torch.cuda.synchronize()
        for s in range(n_steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # L2 flush outside the timed events
                ev[s][0].record(stream)
            g.sample_pass_async(N, it0 + s, res[s].data_ptr())
            g.refine_grids()
            g.update_alpha()
            with torch.cuda.stream(stream):
                ev[s][1].record(stream)
        stream.synchronize()
        for a, b in ev:
            ms.append(a.elapsed_time(b))
        rows = res.cpu().numpy()
        if rows[:, 8].any():
            raise RuntimeError("a timed pass raised a device error flag")
        last = types.SimpleNamespace(**dict(zip(
            ("integral", "variance", "w_max", "efficiency", "n_calls", "combined", "combined_sigma", "chi2_dof"),
            (float(v) for v in rows[-1, :8]))))
        return ms, int(rows[:, 4].sum()), last

    def graph_steps(g, n_steps, it0):
        """The same adaptation iterations captured once as a CUDA graph (L2
        flush, asynchronous pass, rebinning, α update per iteration) and
        replayed; returns per-step ms (total / steps), calls and the last
        pass's result."""
        res = torch.zeros((n_steps, 9), dtype=torch.float64, device=dev)
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            for s in range(n_steps):
                flush.zero_()  # L2 flush between iterations (inside the timed replay)
                g.sample_pass_async(N, it0 + s, res[s].data_ptr())
                g.refine_grids()
                g.update_alpha()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            graph.replay()
            e1.record(stream)
        stream.synchronize()
        total = e0.elapsed_time(e1)
        rows = res.cpu().numpy()
        if rows[:, 8].any():
            raise RuntimeError("a replayed pass raised a device error flag")
        last = types.SimpleNamespace(**dict(zip(
            ("integral", "variance", "w_max", "efficiency", "n_calls", "combined", "combined_sigma", "chi2_dof"),
            (float(v) for v in rows[-1, :8]))))
        del graph
        return [total / n_steps] * n_steps, int(rows[:, 4].sum()), last

    # ---- FP32-eval: headline -------------------------------------------------
    g = V.Vamp(pr, precision=V.PREC_FP32_EVAL, stream=stream)
    it = 0
    for _ in range(args.warmup):
        g.sample_pass(N, it)
        g.refine_grids()
        g.update_alpha()
        it += 1
    stream.synchronize()
    blob = g.checkpoint()  # the state after the warm-up iterations
    # per-pass kernel timing (roofline): the timed iterations, event-timed
    g.profile(True)
    timed_steps(g, args.steps, it, 1)
    ks = g.kernel_stats()
    g.profile(False)
    # headline: the same iterations again from the same state, as one
    # replayed CUDA graph
    g.restore(blob)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ms, calls, last = graph_steps(g, args.steps, it)
    it += args.steps
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t_tot = sum(ms)
    t_max, calls_all = job_throughput(t_tot, float(calls), ws, dev)
    value = calls_all / (t_max / 1e3)
    g.profile(False)

    # ---- unweighted events from the adapted grids (1e6 events) ---------------
    n_ev = pr.n_events
    rb = V.record_bytes(pr.d)
    rec = torch.empty(n_ev * rb, dtype=torch.uint8, device=dev)
    g.generate(1000, rec.data_ptr(), gen_id=0)  # warm-up
    g.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        flush.zero_()
        e0.record(stream)
    gst = g.generate(n_ev, rec.data_ptr(), gen_id=1)
    with torch.cuda.stream(stream):
        e1.record(stream)
    stream.synchronize()
    gen_ms = e0.elapsed_time(e1)
    gks = g.kernel_stats()
    g.profile(False)

    # ---- e2e through host buffers ---------------------------------------------
    K, d, n = pr.n_channels, pr.d, pr.n_bins
    h_edges = torch.empty(K * d * (n + 1), dtype=torch.float64, pin_memory=True).numpy().reshape(K, d, n + 1)
    h_alpha = torch.empty(K, dtype=torch.float64, pin_memory=True).numpy()
    h_shift = torch.empty(K, dtype=torch.float64, pin_memory=True).numpy()
    hbuf = {"edges": h_edges, "alpha": h_alpha, "shift": h_shift}
    wmax = g.get_state(out=hbuf)["w_max"]
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_calls = 0
    for s in range(e2e_steps):
        g.set_state(h_edges, h_alpha, h_shift, wmax)
        r = g.sample_pass(N, it)
        g.refine_grids()
        g.update_alpha()
        wmax = g.get_state(out=hbuf)["w_max"]  # device -> the same pinned buffers
        e2e_calls += r.n_calls
        it += 1
    e2e_t = time.perf_counter() - t0
    bytes_state = 8 * (K * d * (n + 1) + 2 * K + 1)
    e2e = {"value": e2e_calls * ws / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state + 64}

    # ---- FP64 path (same workload, same launch shape) --------------------------
    g64 = V.Vamp(pr, precision=V.PREC_FP64, stream=stream)
    st = g.get_state()
    g64.set_state(st["edges"], st["alpha"], st["shift"], st["w_max"])
    r64 = g64.sample_pass(N, it)
    stream.synchronize()
    # FP32-eval against FP64 on the same grids, α and random stream: the pass
    # integral, and per call the inverse-lookup bins (flips) and weights
    r32 = g.sample_pass(N, it)
    ns = 4096
    e32, e64 = g.eval_calls(0, it, 0, ns), g64.eval_calls(0, it, 0, ns)
    ok = (e32["bins"] >= 0) & (e64["bins"] >= 0)
    flips = int(np.sum(ok & (e32["bins"] != e64["bins"])))
    wrel = np.abs(e32["w"] - e64["w"]) / np.maximum(np.abs(e64["w"]), 1e-300)
    fp32_acc = {"integral_fp32": r32.integral, "integral_fp64": r64.integral,
                "integral_rel_dev": abs(r32.integral - r64.integral) / abs(r64.integral),
                "integral_dev_sigma": abs(r32.integral - r64.integral) / math.sqrt(max(r64.variance, 1e-300)),
                "sample_calls": ns, "lookups": int(ok.sum()), "bin_flips": flips,
                "bin_flips_per_lookup": flips / max(int(ok.sum()), 1),
                "weight_rel_dev_median": float(np.median(wrel)), "weight_rel_dev_max": float(np.max(wrel))}
    f64_steps = max(1, min(args.steps, 3))
    ms64, calls64, _ = timed_steps(g64, f64_steps, it + 1, 0)
    fp64_rate = calls64 / (sum(ms64) / 1e3)

    # ---- many uneven integrations in one launch; the request stream ----------
    batch = run_batch(V, P, 256, args.batch_iters) if args.batch_iters > 0 else None
    serving = None
    if args.serve_seconds > 0 and rank == 0:
        cap = 64 << 20
        serving = {"fp32_eval": run_serving(V, P, torch, dev, V.PREC_FP32_EVAL, args.serve_rate, args.serve_seconds,
                                            120 * 10**9, args.serve_slots, 10, cap)}
        if args.serve_seconds_fp64 > 0:
            serving["fp64"] = run_serving(V, P, torch, dev, V.PREC_FP64, args.serve_rate_fp64,
                                          args.serve_seconds_fp64, 120 * 10**9, args.serve_slots, 10, cap)
        serving["generation_call_limit"] = cap

    # ---- roofline of the dominant kernel (FP32-eval sampling kernel) ----------
    # per pipe: the method's own work per call x calls per second of the
    # kernel, against that pipe's throughput measured on this GPU
    # (vamp_measure_peaks); the binding pipe's fraction is `frac`
    mp = V.measure_peaks()
    k_ms = ks["sample_ms"] / max(ks["sample_launches"], 1)
    kcalls = calls / max(args.steps, 1) / (k_ms / 1e3)  # calls/s of the pass kernel
    kname = g.kernel_name()
    union = kernel_family(kname) == "k_union"
    work = {"alu": (algorithmic_ops_per_call(pr), mp["fp32_lane_ops"], "Tops/s",
                    "32-bit lane-operations (FP32 and integer) per call: the method's work, as for every kernel")}
    if union:
        work["l2"] = (union_l2_bytes_per_call(pr), mp["l2_read_bytes"], "TB/s",
                      "bytes read from L2 per call (a 256-byte density row and a cell entry per coordinate)")
        work["lsu"] = (union_lsu_wavefronts_per_call(pr), mp["lds_wavefronts"], "Twavefronts/s",
                       "shared-memory wavefronts per call (channel records, coordinates, interval broadcasts, "
                       "channel factors)")
        work["xu"] = (union_xu_ops_per_call(pr), mp["xu_lane_ops"], "Tops/s", "MUFU operations per call")
    else:
        work["lsu"] = (lsu_wavefronts_per_call(pr), mp["lds_wavefronts"], "Twavefronts/s",
                       "shared-memory load wavefronts per call (three 4-byte reads per lookup, 32 lanes each)")
        work["xu"] = (xu_ops_per_call(pr), mp["xu_lane_ops"], "Tops/s", "MUFU operations per call")
    work["fp64"] = (fp64_ops_per_call(pr), mp["fp64_lane_ops"], "Tops/s", "FP64 operations per call")
    pipes = {}
    for name, (per_call, peak, unit, what) in work.items():
        ach = per_call * kcalls
        pipes[name] = {"achieved": ach / 1e12, "peak": peak / 1e12, "unit": unit, "frac": ach / peak,
                       "per_call": per_call, "work": what}
    bound = max(pipes, key=lambda k: pipes[k]["frac"])
    bp = pipes[bound]
    roof = {"bound": bound, "achieved": bp["achieved"], "peak": bp["peak"], "unit": bp["unit"],
            "frac": bp["frac"], "traffic": measured_traffic(kname),
            "kernel": kname, "kernel_ms": k_ms, "ops_per_call": algorithmic_ops_per_call(pr),
            "frac_lookups_only": lookup_ops_per_call(pr) * kcalls / mp["fp32_lane_ops"],
            "pipes": pipes,
            "peak_source": "measured on this GPU by vamp_measure_peaks (FFMA, DFMA, MUFU, conflict-free "
                           "shared-load and L2-read kernels)"}
    if batch is not None:
        for tag in ("tuned", "fixed"):
            batch[tag]["frac_of_alu_peak"] = batch[tag]["alu_ops_per_s"] / mp["fp32_lane_ops"]
    # the FP64 form: its floating-point operations against the measured FP64
    # FMA lane rate (the binding pipe), and its 32-bit lane work against the
    # FP32 lane rate
    fp64_ops = fp64_form_ops_per_call(pr) * fp64_rate
    fp64_roof = {"bound": "fp64", "achieved": fp64_ops / 1e12, "peak": mp["fp64_lane_ops"] / 1e12,
                 "unit": "Tops/s", "frac": fp64_ops / mp["fp64_lane_ops"],
                 "ops_per_call": fp64_form_ops_per_call(pr),
                 "frac_alu": algorithmic_ops_per_call(pr) * fp64_rate / mp["fp32_lane_ops"],
                 "peak_source": "measured on this GPU by vamp_measure_peaks (DFMA kernel)"}

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32-eval/f64-accumulate", "data": "synthetic",
           "config": {"workload": WORKLOAD, "calls_per_step": calls / args.steps,
                      "parallelism": f"replicas{ws}", "l2": "flushed (256 MB write) before each iteration, inside the timed graph replay",
                      "timing": "the timed iterations captured once as a CUDA graph and replayed (CUDA events around "
                                "the replay); kernel times for the roofline from an event-timed run of the same "
                                "iterations from the same state",
                      "precision": "FP32-eval"},
           "fp64_path": {"value": fp64_rate, "unit": UNIT, "speedup_fp32_eval": value / ws / fp64_rate,
                         "roofline": fp64_roof},
           "measured_peaks": mp,
           "fp32_accuracy": fp32_acc,
           "generation": {"events": gst["n_written"], "events_per_s": gst["n_written"] / (gen_ms / 1e3),
                          "calls_used": gst["n_calls_used"], "overweight": gst["n_overweight"],
                          "gen_kernel_ms": gks["gen_ms"], "batches": gks["gen_launches"]},
           "last_pass": {"integral": last.integral, "sigma": math.sqrt(max(last.variance, 0.0)),
                         "efficiency": last.efficiency, "combined": last.combined,
                         "combined_sigma": last.combined_sigma, "chi2_dof": last.chi2_dof},
           "e2e": e2e, "gpu_launches": (KERNELS_PER_STEP + (UNION_EXTRA_KERNELS if union else 0)) * args.steps,
           "roofline": roof, "clocks": clk}
    if batch is not None:
        res["batch"] = batch
    if serving is not None:
        res["serving"] = serving
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        thr = os.cpu_count() or 1
        v, ncall, dt = cpu_oracle_rate(base, args.cpu_seconds, thr)
        v1, ncall1, dt1 = cpu_oracle_rate(base, args.cpu_seconds / 4, 1)
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle",
                               "sample": f"one oracle pass of {ncall} calls of the same workload ({dt:.1f} s)",
                               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                                 "sample": f"one oracle pass of {ncall1} calls ({dt1:.1f} s)"}}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)  # with 3 warm-up steps: the 15 iterations of the workload
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch-iters", type=int, default=3, help="timed iterations of the 256-instance batch (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window of the request stream (0: skip)")
    ap.add_argument("--serve-seconds-fp64", type=float, default=60.0, help="arrival window for the FP64 form")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-rate-fp64", type=float, default=16.0,
                    help="offered rate of the FP64 form (below the rate it sustains)")
    ap.add_argument("--serve-slots", type=int, default=256)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

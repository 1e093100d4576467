"""Thin ctypes binding of the C ABI in ``include/vamp.h``.

Argument marshalling only: every step of the integration runs in the CUDA
kernels of ``libvamp_gb300.so``.  There is no CPU fallback -- if the library
is missing or no GPU is present, :func:`load` raises.

PyTorch is used only for device memory (event-record buffers) and streams.

A typical run (the adaptation loop of §3.5, then unweighted events)::

    from paper_1811_09711_gb300 import problems, vamp
    pr = problems.collider()
    g = vamp.Vamp(pr, precision=vamp.PREC_FP32_EVAL)
    for it in range(pr.iterations):
        r = g.sample_pass(pr.calls, it)   # estimate, variance, w_max (Eqs. 23, 31)
        g.refine_grids()                  # rebinning (Eqs. 14, 15)
        g.update_alpha()                  # channel weights (Eq. 25)
    p, w, stats = g.generate_torch(10_000)   # unweighted events (§2)

Many problems at once: :class:`Batch`; a request stream: :class:`Server`;
graph-capturable iterations: :meth:`Vamp.sample_pass_async`.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

VAMP_OK, VAMP_ERR_INVALID_ARG, VAMP_ERR_OOM, VAMP_ERR_CUDA, VAMP_ERR_TIMEOUT, \
    VAMP_ERR_NUMERIC, VAMP_ERR_STATE, VAMP_ERR_LIMIT = range(8)
PREC_FP64, PREC_FP32_EVAL = 0, 1

_lock = threading.Lock()
_lib = None


class VampError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "VAMP_OK", 1: "VAMP_ERR_INVALID_ARG", 2: "VAMP_ERR_OOM", 3: "VAMP_ERR_CUDA",
           4: "VAMP_ERR_TIMEOUT", 5: "VAMP_ERR_NUMERIC", 6: "VAMP_ERR_STATE",
           7: "VAMP_ERR_LIMIT"}


class MapDesc(C.Structure):
    _fields_ = [("n_mapped", C.c_int32), ("coord", C.c_int32 * 4), ("kind", C.c_int32 * 4),
                ("a", C.c_double * 4), ("b", C.c_double * 4)]


class Config(C.Structure):
    _fields_ = [
        ("d", C.c_int32), ("n_channels", C.c_int32), ("n_bins", C.c_int32),
        ("channels", C.POINTER(MapDesc)),
        ("n_peaks", C.c_int32),
        ("peak_weight", C.POINTER(C.c_double)),
        ("peaks", C.POINTER(MapDesc)),
        ("gauss_sigma", C.c_double), ("gauss_centre", C.c_double), ("gauss_norm", C.c_int32),
        ("seed", C.c_uint64), ("request_id", C.c_uint32),
        ("grid_alpha", C.c_double), ("beta", C.c_double), ("n_min", C.c_int64),
        ("smooth", C.c_int32), ("omega_mode", C.c_int32),
        ("gen_batch", C.c_int64), ("combine_from", C.c_int32), ("precision", C.c_int32),
        ("stratified", C.c_int32),
        ("n_equiv", C.c_int32), ("equiv", C.POINTER(C.c_int32)),
    ]


class PassResult(C.Structure):
    _fields_ = [("integral", C.c_double), ("variance", C.c_double), ("w_max", C.c_double),
                ("efficiency", C.c_double), ("n_calls", C.c_int64), ("combined", C.c_double),
                ("combined_sigma", C.c_double), ("chi2_dof", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    def __repr__(self):
        return f"PassResult({self.as_dict()})"


class PipePeaks(C.Structure):
    _fields_ = [("fp32_lane_ops", C.c_double), ("fp64_lane_ops", C.c_double), ("xu_lane_ops", C.c_double),
                ("lds_wavefronts", C.c_double), ("l2_read_bytes", C.c_double)]


class RequestResult(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int32), ("iterations", C.c_int32),
                ("result", PassResult), ("calls_total", C.c_int64), ("events_written", C.c_int64),
                ("events_calls_used", C.c_int64), ("events_overweight", C.c_int64),
                ("queue_s", C.c_double), ("latency_s", C.c_double)]


def load():
    """Build (if the sources changed since the last build) and load the CUDA
    library; raise if it is unusable or was not built from these sources."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build(force=bool(os.environ.get("VAMP_REBUILD")))
        lib = C.CDLL(path)
        lib.vamp_source_hash.argtypes = []
        lib.vamp_source_hash.restype = C.c_char_p
        built_from, current = lib.vamp_source_hash().decode(), _build.source_hash()
        if built_from != current:
            raise RuntimeError(f"{path} was built from other sources (hash {built_from[:16]}, "
                               f"sources {current[:16]}); rebuild with VAMP_REBUILD=1")
        vp, i32, i64, u32, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
        st = C.c_int
        lib.vamp_create.argtypes = [C.POINTER(Config), vp, C.POINTER(vp)]
        lib.vamp_create.restype = st
        lib.vamp_sample_pass.argtypes = [vp, i64, u32, C.POINTER(PassResult)]
        lib.vamp_sample_pass.restype = st
        lib.vamp_sample_pass_async.argtypes = [vp, i64, u32, vp]
        lib.vamp_sample_pass_async.restype = st
        lib.vamp_refine_grids.argtypes = [vp]
        lib.vamp_refine_grids.restype = st
        lib.vamp_update_alpha.argtypes = [vp]
        lib.vamp_update_alpha.restype = st
        lib.vamp_generate.argtypes = [vp, i64, u32, vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        lib.vamp_generate.restype = st
        lib.vamp_record_bytes.argtypes = [i32]
        lib.vamp_record_bytes.restype = i64
        lib.vamp_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(dbl)]
        lib.vamp_get_state.restype = st
        lib.vamp_set_state.argtypes = [vp, vp, vp, vp, dbl]
        lib.vamp_set_state.restype = st
        lib.vamp_get_pass.argtypes = [vp, vp, vp, vp, vp]
        lib.vamp_get_pass.restype = st
        lib.vamp_eval_calls.argtypes = [vp, i32, u32, u32, i32, vp, vp, vp, vp, vp]
        lib.vamp_eval_calls.restype = st
        lib.vamp_allocate.argtypes = [vp, i64, C.POINTER(i64)]
        lib.vamp_allocate.restype = st
        lib.vamp_profile.argtypes = [vp, i32]
        lib.vamp_profile.restype = st
        lib.vamp_kernel_stats.argtypes = [vp, C.POINTER(dbl), C.POINTER(i64), C.POINTER(dbl), C.POINTER(i64)]
        lib.vamp_kernel_stats.restype = st
        lib.vamp_sample_pass_static.argtypes = [C.POINTER(Config), vp, vp, vp, i64, u32, vp, vp,
                                                C.POINTER(PassResult), C.c_char_p, i32]
        lib.vamp_sample_pass_static.restype = st
        lib.vamp_pass_kernel_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                                C.POINTER(i32), C.POINTER(i32)]
        lib.vamp_pass_kernel_info.restype = st
        lib.vamp_measure_peaks.argtypes = [C.POINTER(PipePeaks)]
        lib.vamp_measure_peaks.restype = st
        lib.vamp_pass_kernel_name.argtypes = [vp, i32, C.c_char_p, i32]
        lib.vamp_pass_kernel_name.restype = st
        lib.vamp_pass_kernel_candidates.argtypes = [vp, C.POINTER(i32)]
        lib.vamp_pass_kernel_candidates.restype = st
        lib.vamp_select_pass_kernel.argtypes = [vp, i32]
        lib.vamp_select_pass_kernel.restype = st
        lib.vamp_batch_create.argtypes = [C.POINTER(Config), i32, i32, C.POINTER(vp)]
        lib.vamp_batch_create.restype = st
        lib.vamp_batch_iterate.argtypes = [vp, vp, u32, i32, C.POINTER(PassResult)]
        lib.vamp_batch_iterate.restype = st
        lib.vamp_batch_get_state.argtypes = [vp, i32, vp, vp, vp, C.POINTER(dbl)]
        lib.vamp_batch_get_state.restype = st
        lib.vamp_batch_tuning.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(dbl), C.POINTER(dbl)]
        lib.vamp_batch_tuning.restype = st
        lib.vamp_batch_destroy.argtypes = [vp]
        lib.vamp_batch_destroy.restype = None
        lib.vamp_batch_last_error.argtypes = [vp]
        lib.vamp_batch_last_error.restype = C.c_char_p
        lib.vamp_server_create.argtypes = [i32, i64, i32, C.POINTER(vp)]
        lib.vamp_server_create.restype = st
        lib.vamp_server_submit.argtypes = [vp, C.POINTER(Config), i32, i64, i64, i64, vp, C.POINTER(C.c_uint64)]
        lib.vamp_server_submit.restype = st
        lib.vamp_server_submit_state.argtypes = [vp, C.POINTER(Config), i32, i64, i64, i64, vp, vp,
                                                 C.POINTER(C.c_uint64)]
        lib.vamp_server_submit_state.restype = st
        lib.vamp_server_poll.argtypes = [vp, C.POINTER(RequestResult), i32]
        lib.vamp_server_poll.restype = i32
        lib.vamp_server_wait_idle.argtypes = [vp, dbl]
        lib.vamp_server_wait_idle.restype = st
        lib.vamp_server_stats.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        lib.vamp_server_stats.restype = st
        lib.vamp_server_load.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)]
        lib.vamp_server_load.restype = st
        lib.vamp_server_destroy.argtypes = [vp]
        lib.vamp_server_destroy.restype = None
        lib.vamp_checkpoint_bytes.argtypes = [vp]
        lib.vamp_checkpoint_bytes.restype = i64
        lib.vamp_checkpoint.argtypes = [vp, vp, i64]
        lib.vamp_checkpoint.restype = st
        lib.vamp_restore.argtypes = [vp, vp, i64]
        lib.vamp_restore.restype = st
        lib.vamp_selftest_bounded_wait.argtypes = [i64, C.POINTER(i64)]
        lib.vamp_selftest_bounded_wait.restype = st
        lib.vamp_destroy.argtypes = [vp]
        lib.vamp_destroy.restype = None
        lib.vamp_last_error.argtypes = [vp]
        lib.vamp_last_error.restype = C.c_char_p
        lib.vamp_status_string.argtypes = [st]
        lib.vamp_status_string.restype = C.c_char_p
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _map_array(ms) -> C.Array:
    arr = (MapDesc * len(ms))()
    for q in range(len(ms)):
        r = arr[q]
        r.n_mapped = int(ms.n_mapped[q])
        for s in range(4):
            r.coord[s] = int(ms.coord[q, s])
            r.kind[s] = int(ms.kind[q, s])
            r.a[s] = float(ms.a[q, s])
            r.b[s] = float(ms.b[q, s])
    return arr


def make_config(problem, precision: int = PREC_FP64):
    """vamp_config for a problem (see ``problems.Problem``); returns the
    struct and the host arrays it points into (keep both alive)."""
    ch = _map_array(problem.channels)
    pk = _map_array(problem.peaks)
    w = np.ascontiguousarray(problem.peak_weight, np.float64)
    eq = getattr(problem, "equivalences", None)
    eq = (np.zeros((0, 2 + 2 * int(problem.d)), np.int32) if eq is None
          else np.ascontiguousarray(eq, np.int32).reshape(-1, 2 + 2 * int(problem.d)))
    cfg = Config(int(problem.d), int(problem.n_channels), int(problem.n_bins),
                 C.cast(ch, C.POINTER(MapDesc)), int(problem.n_peaks),
                 w.ctypes.data_as(C.POINTER(C.c_double)), C.cast(pk, C.POINTER(MapDesc)),
                 float(problem.gauss_sigma), float(problem.gauss_centre), int(problem.gauss_norm),
                 int(problem.seed) & (2**64 - 1), int(problem.request_id) & 0xffffffff,
                 float(problem.grid_alpha), float(problem.beta), int(problem.n_min),
                 int(problem.smooth), int(problem.omega_mode), int(problem.gen_batch),
                 int(problem.combine_from), int(precision), int(getattr(problem, "stratified", 0)),
                 int(eq.shape[0]), eq.ctypes.data_as(C.POINTER(C.c_int32)) if eq.shape[0] else None)
    return cfg, (ch, pk, w, eq)


def source_hash() -> str:
    """Hash of the sources the loaded library was built from (vamp_source_hash)."""
    return load().vamp_source_hash().decode()


def record_bytes(d: int) -> int:
    return int(load().vamp_record_bytes(int(d)))


class Vamp:
    """One integration context on the current CUDA device.

    ``stream``: a ``torch.cuda.Stream`` (or an integer cudaStream_t, or None
    for the legacy default stream).
    """

    def __init__(self, problem, precision: int = PREC_FP64, stream=None):
        self.lib = load()
        self.problem = problem
        self.d, self.K, self.n = int(problem.d), int(problem.n_channels), int(problem.n_bins)
        self.precision = precision
        if stream is not None and hasattr(stream, "cuda_stream"):
            self._stream_obj = stream
            stream = stream.cuda_stream
        self.stream = int(stream or 0)
        cfg, keep = make_config(problem, precision)
        h = C.c_void_p()
        rc = self.lib.vamp_create(C.byref(cfg), C.c_void_p(self.stream), C.byref(h))
        if rc != VAMP_OK:
            raise VampError(rc, "vamp_create failed")
        self.h = h

    def _check(self, rc):
        if rc != VAMP_OK:
            raise VampError(rc, self.lib.vamp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.vamp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- hot path ----------------------------------------------------------
    def sample_pass(self, n_calls: int, iteration: int) -> PassResult:
        out = PassResult()
        self._check(self.lib.vamp_sample_pass(self.h, int(n_calls), int(iteration), C.byref(out)))
        return out

    def sample_pass_async(self, n_calls: int, iteration: int, dev_out_ptr: int):
        """vamp_sample_pass_async: enqueues the pass; 9 doubles land at the
        device address dev_out_ptr (integral, variance, w_max, efficiency,
        n_calls, combined, combined_sigma, chi2_dof, error flags)."""
        self._check(self.lib.vamp_sample_pass_async(self.h, int(n_calls), int(iteration), C.c_void_p(dev_out_ptr)))

    def refine_grids(self):
        self._check(self.lib.vamp_refine_grids(self.h))

    def update_alpha(self):
        self._check(self.lib.vamp_update_alpha(self.h))

    def generate(self, n_events: int, records_ptr: int, gen_id: int = 0):
        """Writes up to n_events records to device memory at records_ptr."""
        nw, nu, no = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self.lib.vamp_generate(self.h, int(n_events), int(gen_id), C.c_void_p(records_ptr),
                                           C.byref(nw), C.byref(nu), C.byref(no)))
        return {"n_written": nw.value, "n_calls_used": nu.value, "n_overweight": no.value}

    def generate_torch(self, n_events: int, gen_id: int = 0, out=None):
        """generate() into a torch uint8 device tensor; returns (p, w, stats)
        decoded on the host (p: float32 [n, d], w: float64 [n])."""
        import torch
        rb = record_bytes(self.d)
        if out is None:
            out = torch.empty(max(n_events, 1) * rb, dtype=torch.uint8, device="cuda")
        st = self.generate(n_events, out.data_ptr(), gen_id)
        raw = out[: st["n_written"] * rb].cpu().numpy()
        return decode_records(raw, self.d) + (st,)

    # -- kernel timing ---------------------------------------------------------
    def profile(self, enable: bool = True):
        self._check(self.lib.vamp_profile(self.h, int(bool(enable))))

    def kernel_stats(self):
        sm, sn, gm, gn = C.c_double(), C.c_int64(), C.c_double(), C.c_int64()
        self._check(self.lib.vamp_kernel_stats(self.h, C.byref(sm), C.byref(sn), C.byref(gm), C.byref(gn)))
        return {"sample_ms": sm.value, "sample_launches": sn.value, "gen_ms": gm.value,
                "gen_launches": gn.value}

    def kernel_info(self):
        f, c, dd, nn, mb = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self.lib.vamp_pass_kernel_info(self.h, C.byref(f), C.byref(c), C.byref(dd), C.byref(nn),
                                                   C.byref(mb)))
        return {"fp32": f.value, "calls_per_thread": c.value, "shape_d": dd.value, "shape_n": nn.value,
                "ctas_per_sm": mb.value}

    def kernel_name(self, mode: int = 0) -> str:
        """Name of the pass kernel as profilers print it (vamp_pass_kernel_name)."""
        buf = C.create_string_buffer(128)
        self._check(self.lib.vamp_pass_kernel_name(self.h, int(mode), buf, 128))
        return buf.value.decode()

    def kernel_candidates(self) -> int:
        """Number of compiled pass kernels that can run this problem (vamp_pass_kernel_candidates)."""
        n = C.c_int32()
        self._check(self.lib.vamp_pass_kernel_candidates(self.h, C.byref(n)))
        return n.value

    def select_kernel(self, index: int):
        """Pin the pass kernel to candidate `index` (vamp_select_pass_kernel)."""
        self._check(self.lib.vamp_select_pass_kernel(self.h, int(index)))

    def select_family(self, family: str) -> str:
        """Pin the pass kernel to the first candidate of a kernel family
        ("k_pass": the channel loop per call, whose FP32-eval arithmetic the
        batch and server kernels share; "k_union": the pass over
        per-coordinate interval tables); returns its name."""
        for i in range(self.kernel_candidates()):
            self.select_kernel(i)
            name = self.kernel_name(0)
            if name.startswith(family + "<"):
                return name
        raise VampError(VAMP_ERR_INVALID_ARG, f"no {family} kernel for this problem")

    # -- state ---------------------------------------------------------------
    def get_state(self, out=None):
        """Grids, α, shifts and w_max (vamp_get_state).  ``out``: optional dict
        of C-contiguous float64 arrays "edges" [K, d, n+1], "alpha" [K] and
        "shift" [K] to fill in place (pinned host memory avoids a staging copy)."""
        shapes = {"edges": (self.K, self.d, self.n + 1), "alpha": (self.K,), "shift": (self.K,)}
        if out is None:
            out = {k: np.zeros(v, np.float64) for k, v in shapes.items()}
        for k, v in shapes.items():
            arr = out[k]
            if arr.dtype != np.float64 or arr.shape != v or not arr.flags.c_contiguous:
                raise ValueError(f"out[{k!r}] must be a C-contiguous float64 array of shape {v}")
        e, a, s = out["edges"], out["alpha"], out["shift"]
        wm = C.c_double()
        self._check(self.lib.vamp_get_state(self.h, _ptr(e), _ptr(a), _ptr(s), C.byref(wm)))
        return {"edges": e, "alpha": a, "shift": s, "w_max": wm.value}

    def set_state(self, edges=None, alpha=None, shift=None, w_max: float = 0.0):
        e = None if edges is None else np.ascontiguousarray(edges, np.float64)
        a = None if alpha is None else np.ascontiguousarray(alpha, np.float64)
        s = None if shift is None else np.ascontiguousarray(shift, np.float64)
        self._check(self.lib.vamp_set_state(self.h, _ptr(e), _ptr(a), _ptr(s), float(w_max)))

    def checkpoint(self) -> bytes:
        """The adaptation state as a self-describing blob (vamp_checkpoint)."""
        n = int(self.lib.vamp_checkpoint_bytes(self.h))
        if n < 0:
            raise VampError(VAMP_ERR_CUDA, self.lib.vamp_last_error(self.h).decode())
        buf = C.create_string_buffer(n)
        self._check(self.lib.vamp_checkpoint(self.h, buf, n))
        return buf.raw

    def restore(self, blob: bytes):
        buf = C.create_string_buffer(bytes(blob), len(blob))
        self._check(self.lib.vamp_restore(self.h, buf, len(blob)))

    def get_pass(self):
        D = np.zeros((self.K, self.d, self.n), np.float64)
        Ic = np.zeros(self.K, np.float64)
        Vc = np.zeros(self.K, np.float64)
        Nc = np.zeros(self.K, np.int64)
        self._check(self.lib.vamp_get_pass(self.h, _ptr(D), _ptr(Ic), _ptr(Vc), _ptr(Nc)))
        return {"D": D, "Ic": Ic, "Vc": Vc, "Nc": Nc}

    def allocate(self, n_calls: int) -> int:
        t = C.c_int64()
        self._check(self.lib.vamp_allocate(self.h, int(n_calls), C.byref(t)))
        return t.value

    def eval_calls(self, mode: int, field: int, call0: int, count: int, with_bins: bool = True):
        d, K = self.d, self.K
        x = np.zeros((count, d), np.float64)
        p = np.zeros((count, d), np.float64)
        jf = np.zeros((count, d), np.int32)
        bins = np.zeros((count, K, d), np.int32) if with_bins else None
        fgwc = np.zeros((count, 4), np.float64)
        self._check(self.lib.vamp_eval_calls(self.h, int(mode), int(field), int(call0), int(count),
                                             _ptr(x), _ptr(p), _ptr(jf), _ptr(bins), _ptr(fgwc)))
        return {"x": x, "p": p, "jf": jf, "bins": bins, "f": fgwc[:, 0], "g": fgwc[:, 1],
                "w": fgwc[:, 2], "channel": fgwc[:, 3].astype(np.int64)}


class Batch:
    """Many independent integrations advanced together (vamp_batch_*)."""

    def __init__(self, problems, precision: int = PREC_FP32_EVAL, autotune: bool = True):
        self.lib = load()
        self.problems = list(problems)
        cfgs = (Config * len(self.problems))()
        self._keep = []
        for i, pr in enumerate(self.problems):
            cfg, keep = make_config(pr, precision)
            cfgs[i] = cfg
            self._keep.append(keep)
        self._cfgs = cfgs
        h = C.c_void_p()
        rc = self.lib.vamp_batch_create(cfgs, len(self.problems), int(bool(autotune)), C.byref(h))
        if rc != VAMP_OK:
            raise VampError(rc, "vamp_batch_create failed")
        self.h = h
        self.n = len(self.problems)

    def _check(self, rc):
        if rc != VAMP_OK:
            raise VampError(rc, self.lib.vamp_batch_last_error(self.h).decode())

    def iterate(self, n_calls, iteration: int, adapt: int = 3):
        nc = np.ascontiguousarray(n_calls, np.int64)
        res = (PassResult * self.n)()
        self._check(self.lib.vamp_batch_iterate(self.h, _ptr(nc), int(iteration), int(adapt), res))
        return list(res)

    def get_state(self, i: int):
        pr = self.problems[i]
        e = np.zeros((pr.n_channels, pr.d, pr.n_bins + 1), np.float64)
        a = np.zeros(pr.n_channels, np.float64)
        s = np.zeros(pr.n_channels, np.float64)
        wm = C.c_double()
        self._check(self.lib.vamp_batch_get_state(self.h, int(i), _ptr(e), _ptr(a), _ptr(s), C.byref(wm)))
        return {"edges": e, "alpha": a, "shift": s, "w_max": wm.value}

    def tuning(self):
        ic, bk, tm, fm = C.c_int64(), C.c_int32(), C.c_double(), C.c_double()
        self._check(self.lib.vamp_batch_tuning(self.h, C.byref(ic), C.byref(bk), C.byref(tm), C.byref(fm)))
        return {"item_calls": ic.value, "budget_kb": bk.value, "tuned_ms": tm.value, "fixed_ms": fm.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.vamp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (vamp_server_*): submit whole
    integrate-then-generate requests, poll completed ones."""

    def __init__(self, max_slots: int = 64, mem_budget_bytes: int = 8 << 30, precision: int = PREC_FP32_EVAL):
        self.lib = load()
        self.precision = precision
        h = C.c_void_p()
        rc = self.lib.vamp_server_create(int(max_slots), int(mem_budget_bytes), int(precision), C.byref(h))
        if rc != VAMP_OK:
            raise VampError(rc, "vamp_server_create failed")
        self.h = h

    def submit(self, problem, iterations: int, calls: int, n_events: int = 0, records_ptr: int = 0,
               max_gen_calls: int = 0, state_ptr: int = 0) -> int:
        """Queue a request; ``state_ptr`` (device, K*d*(n+1) + 2K float64)
        optionally receives the adapted grids, α and shifts
        (vamp_server_submit_state)."""
        cfg, keep = make_config(problem, self.precision)
        rid = C.c_uint64()
        rc = self.lib.vamp_server_submit_state(self.h, C.byref(cfg), int(iterations), int(calls), int(n_events),
                                               int(max_gen_calls), C.c_void_p(records_ptr or None),
                                               C.c_void_p(state_ptr or None), C.byref(rid))
        del keep  # the server copied the description
        if rc != VAMP_OK:
            raise VampError(rc, "vamp_server_submit rejected the request")
        return rid.value

    def poll(self, max_results: int = 256):
        buf = (RequestResult * max_results)()
        k = self.lib.vamp_server_poll(self.h, buf, int(max_results))
        return [buf[i] for i in range(k)]

    def wait_idle(self, timeout_s: float = 600.0):
        rc = self.lib.vamp_server_wait_idle(self.h, float(timeout_s))
        if rc != VAMP_OK:
            raise VampError(rc, "requests still pending")

    def stats(self):
        t, c, e, m = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self.lib.vamp_server_stats(self.h, C.byref(t), C.byref(c), C.byref(e), C.byref(m))
        return {"ticks": t.value, "calls": c.value, "events": e.value, "mem_in_use": m.value}

    def load(self):
        q, i, g, b = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
        self.lib.vamp_server_load(self.h, C.byref(q), C.byref(i), C.byref(g), C.byref(b))
        return {"queued": q.value, "integrating": i.value, "generating": g.value, "gen_batches": b.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.vamp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_peaks() -> dict:
    """vamp_measure_peaks: measured per-pipe throughput of the current GPU
    (per second, all SMs): FP32 and FP64 FMA lane-instructions, MUFU
    lane-instructions, shared-memory load wavefronts."""
    pk = PipePeaks()
    rc = load().vamp_measure_peaks(C.byref(pk))
    if rc != VAMP_OK:
        raise VampError(rc, "vamp_measure_peaks failed")
    return {k: getattr(pk, k) for k, _ in PipePeaks._fields_}


def selftest_bounded_wait(limit_cycles: int):
    """vamp_selftest_bounded_wait: (status, cycles waited)."""
    lib = load()
    cyc = C.c_int64()
    rc = lib.vamp_selftest_bounded_wait(int(limit_cycles), C.byref(cyc))
    return rc, cyc.value


def sample_pass_static(problem, precision: int, edges_ptr: int, alpha_ptr: int, shift_ptr: int,
                       n_calls: int, iteration: int, stream: int = 0, D_out_ptr: int = 0):
    """vamp_sample_pass_static: one pass whose working memory is the
    library's static device array (no allocation); device pointers in,
    host PassResult out."""
    lib = load()
    cfg, keep = make_config(problem, precision)
    out = PassResult()
    msg = C.create_string_buffer(256)
    rc = lib.vamp_sample_pass_static(C.byref(cfg), C.c_void_p(edges_ptr), C.c_void_p(alpha_ptr),
                                     C.c_void_p(shift_ptr), int(n_calls), int(iteration),
                                     C.c_void_p(stream), C.c_void_p(D_out_ptr or None), C.byref(out),
                                     msg, 256)
    if rc != VAMP_OK:
        raise VampError(rc, msg.value.decode())
    return out


def decode_records(raw: np.ndarray, d: int):
    """Split raw event records into (p float32 [n, d], w float64 [n])."""
    rb = ((4 * d + 7) & ~7) + 8
    n = raw.size // rb
    r = raw[: n * rb].reshape(n, rb)
    p = r[:, : 4 * d].copy().view(np.float32).reshape(n, d)
    w = r[:, rb - 8:].copy().view(np.float64).reshape(n)
    return p, w

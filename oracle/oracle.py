"""ctypes front end of the FP64 CPU oracle (``vamp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` are the only callers.  This module does
not import the CUDA library or its Python binding; a problem is any object
with the attributes of ``paper_1811_09711_gb300.problems.Problem`` (duck
typed), so the oracle and the product share nothing but the seeded input
arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# VAMP_ORACLE_SRC / VAMP_ORACLE_LIB let the mutation tests build a copy of the
# oracle with a planted mistake; normal runs use the committed source.
_SRC = os.environ.get("VAMP_ORACLE_SRC", os.path.join(_HERE, "vamp_oracle.c"))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.environ.get("VAMP_ORACLE_LIB", os.path.join(_LIBDIR, "libvamp_oracle.so"))
_lock = threading.Lock()
_lib = None

OR_OK, OR_ERR_ARG, OR_ERR_STATE, OR_ERR_NUMERIC, OR_ERR_MEM = range(5)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction) into oracle/_lib."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("d", C.c_int32), ("n_channels", C.c_int32), ("n_bins", C.c_int32),
        ("ch_nmap", C.c_void_p), ("ch_coord", C.c_void_p), ("ch_kind", C.c_void_p),
        ("ch_a", C.c_void_p), ("ch_b", C.c_void_p),
        ("n_peaks", C.c_int32),
        ("pk_w", C.c_void_p),
        ("pk_nmap", C.c_void_p), ("pk_coord", C.c_void_p), ("pk_kind", C.c_void_p),
        ("pk_a", C.c_void_p), ("pk_b", C.c_void_p),
        ("gauss_sigma", C.c_double), ("gauss_centre", C.c_double),
        ("gauss_norm", C.c_int32),
        ("seed", C.c_uint64), ("request_id", C.c_uint32),
        ("grid_alpha", C.c_double), ("beta", C.c_double),
        ("n_min", C.c_int64),
        ("smooth", C.c_int32), ("omega_mode", C.c_int32),
        ("gen_batch", C.c_int64),
        ("stratified", C.c_int32),
        ("n_equiv", C.c_int32), ("equiv", C.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            vp, i32, i64, u32, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
            lib.or_create.argtypes = [C.POINTER(_Problem), C.POINTER(C.c_int)]
            lib.or_create.restype = vp
            lib.or_destroy.argtypes = [vp]
            lib.or_destroy.restype = None
            lib.or_philox4x32_10.argtypes = [vp, vp, vp]
            lib.or_philox4x32_10.restype = None
            lib.or_allocate.argtypes = [vp, i64]
            lib.or_allocate.restype = i64
            lib.or_sample_pass.argtypes = [vp, i64, u32, C.c_int, C.c_int, vp]
            lib.or_sample_pass.restype = C.c_int
            lib.or_refine_grids.argtypes = [vp]
            lib.or_refine_grids.restype = C.c_int
            lib.or_update_alpha.argtypes = [vp]
            lib.or_update_alpha.restype = C.c_int
            lib.or_generate.argtypes = [vp, i64, u32, vp, vp, vp]
            lib.or_generate.restype = C.c_int
            lib.or_eval_call.argtypes = [vp, C.c_int, u32, u32, vp, vp, vp, vp, vp, vp]
            lib.or_eval_call.restype = C.c_int
            lib.or_f.argtypes = [vp, vp]
            lib.or_f.restype = dbl
            lib.or_g_point.argtypes = [vp, vp]
            lib.or_g_point.restype = dbl
            lib.or_grid_density.argtypes = [vp, C.c_int, vp]
            lib.or_grid_density.restype = dbl
            lib.or_channel_forward.argtypes = [vp, C.c_int, vp, vp, vp]
            lib.or_channel_forward.restype = None
            lib.or_channel_inverse.argtypes = [vp, C.c_int, vp, vp, vp]
            lib.or_channel_inverse.restype = None
            lib.or_refine_row.argtypes = [vp, C.c_int, C.c_int, dbl, vp]
            lib.or_refine_row.restype = None
            lib.or_get_state.argtypes = [vp, vp, vp, vp, vp]
            lib.or_get_state.restype = None
            lib.or_set_state.argtypes = [vp, vp, vp, vp, dbl, C.c_int]
            lib.or_set_state.restype = None
            lib.or_get_pass.argtypes = [vp, vp, vp, vp, vp]
            lib.or_get_pass.restype = None
            lib.or_alpha_update_raw.argtypes = [C.c_int, vp, vp, vp, vp, dbl, vp]
            lib.or_alpha_update_raw.restype = None
            lib.or_allocate_raw.argtypes = [C.c_int, vp, i64, i64, vp, vp]
            lib.or_allocate_raw.restype = i64
            lib.or_strat_cells_per_axis.argtypes = [i64, C.c_int]
            lib.or_strat_cells_per_axis.restype = i64
            lib.or_get_pooled.argtypes = [vp, vp]
            lib.or_get_pooled.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (oracle implementation)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def refine_row(D, edges, alpha_grid: float = 1.5, smooth: int = 0) -> np.ndarray:
    """Refine one stand-alone grid row (Eqs. 14, 15); returns the new edges."""
    lib = _load()
    D = np.ascontiguousarray(D, dtype=np.float64)
    e = np.array(edges, dtype=np.float64)
    assert e.shape[0] == D.shape[0] + 1
    lib.or_refine_row(_ptr(D), int(D.shape[0]), int(smooth), float(alpha_grid), _ptr(e))
    return e


def alpha_update(alpha, omega, Ic, Nc, beta: float = 0.5) -> np.ndarray:
    """Channel-weight update (Eq. 25) as a pure function of per-channel data."""
    lib = _load()
    a = np.ascontiguousarray(alpha, np.float64)
    om = np.ascontiguousarray(omega, np.float64)
    ic = np.ascontiguousarray(Ic, np.float64)
    nc = np.ascontiguousarray(Nc, np.int64)
    out = np.zeros_like(a)
    lib.or_alpha_update_raw(int(a.shape[0]), _ptr(a), _ptr(om), _ptr(ic), _ptr(nc), float(beta),
                            _ptr(out))
    return out


def strat_cells_per_axis(n_calls: int, d: int) -> int:
    """R16: the largest m (<= 2^20) with 2 m^d <= n_calls."""
    return int(_load().or_strat_cells_per_axis(int(n_calls), int(d)))


def allocate(alpha, n_calls: int, n_min: int = 10):
    """Integer calls per channel and their exclusive prefix (reading of §3.4)."""
    lib = _load()
    a = np.ascontiguousarray(alpha, np.float64)
    nc = np.zeros(a.shape[0], np.int64)
    pc = np.zeros(a.shape[0] + 1, np.int64)
    lib.or_allocate_raw(int(a.shape[0]), _ptr(a), int(n_calls), int(n_min), _ptr(nc), _ptr(pc))
    return nc, pc


class PassResult:
    __slots__ = ("integral", "variance", "w_max", "efficiency", "n_calls", "combined",
                 "combined_sigma", "chi2_dof")

    def __init__(self, v):
        (self.integral, self.variance, self.w_max, self.efficiency, n, self.combined,
         self.combined_sigma, self.chi2_dof) = [float(t) for t in v]
        self.n_calls = int(n)

    def as_dict(self):
        return {k: getattr(self, k) for k in self.__slots__}

    def __repr__(self):
        return f"PassResult({self.as_dict()})"


class Oracle:
    """One oracle integration context for a problem (FP64, CPU)."""

    def __init__(self, problem):
        self.lib = _load()
        pr = problem
        self.d, self.K, self.n = int(pr.d), int(pr.n_channels), int(pr.n_bins)
        self.P = int(pr.n_peaks)
        ch, pk = pr.channels, pr.peaks
        self._keep = [
            np.ascontiguousarray(ch.n_mapped, np.int32), np.ascontiguousarray(ch.coord, np.int32),
            np.ascontiguousarray(ch.kind, np.int32), np.ascontiguousarray(ch.a, np.float64),
            np.ascontiguousarray(ch.b, np.float64),
            np.ascontiguousarray(pr.peak_weight, np.float64),
            np.ascontiguousarray(pk.n_mapped, np.int32), np.ascontiguousarray(pk.coord, np.int32),
            np.ascontiguousarray(pk.kind, np.int32), np.ascontiguousarray(pk.a, np.float64),
            np.ascontiguousarray(pk.b, np.float64),
        ]
        eq = getattr(pr, "equivalences", None)
        eq = np.zeros((0, 2 + 2 * self.d), np.int32) if eq is None else np.ascontiguousarray(eq, np.int32)
        self._keep.append(eq)
        k = self._keep
        st = _Problem(self.d, self.K, self.n, _ptr(k[0]).value, _ptr(k[1]).value, _ptr(k[2]).value,
                      _ptr(k[3]).value, _ptr(k[4]).value, self.P, _ptr(k[5]).value,
                      _ptr(k[6]).value, _ptr(k[7]).value, _ptr(k[8]).value, _ptr(k[9]).value,
                      _ptr(k[10]).value, float(pr.gauss_sigma), float(pr.gauss_centre),
                      int(pr.gauss_norm), int(pr.seed) & (2**64 - 1), int(pr.request_id),
                      float(pr.grid_alpha), float(pr.beta), int(pr.n_min), int(pr.smooth),
                      int(pr.omega_mode), int(pr.gen_batch), int(getattr(pr, "stratified", 0)),
                      int(eq.shape[0]), _ptr(eq).value if eq.shape[0] else None)
        status = C.c_int(0)
        self.h = self.lib.or_create(C.byref(st), C.byref(status))
        if not self.h:
            raise ValueError(f"oracle rejected the problem (status {status.value})")

    def close(self):
        if getattr(self, "h", None):
            self.lib.or_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the integration loop -------------------------------------------
    def allocate(self, n_calls: int) -> int:
        return int(self.lib.or_allocate(self.h, int(n_calls)))

    def sample_pass(self, n_calls: int, iteration: int, combine: bool = False,
                    n_threads: int = 1) -> PassResult:
        out = np.zeros(8, np.float64)
        rc = self.lib.or_sample_pass(self.h, int(n_calls), int(iteration), int(bool(combine)),
                                     int(n_threads), _ptr(out))
        if rc != OR_OK:
            raise RuntimeError(f"oracle sample_pass failed ({rc})")
        return PassResult(out)

    def refine_grids(self):
        rc = self.lib.or_refine_grids(self.h)
        if rc != OR_OK:
            raise RuntimeError(f"oracle refine failed ({rc})")

    def update_alpha(self):
        rc = self.lib.or_update_alpha(self.h)
        if rc != OR_OK:
            raise RuntimeError(f"oracle alpha update failed ({rc})")

    def generate(self, n_events: int, gen_id: int = 0):
        p = np.zeros((max(n_events, 1), self.d), np.float32)
        w = np.zeros(max(n_events, 1), np.float64)
        st = np.zeros(4, np.int64)
        rc = self.lib.or_generate(self.h, int(n_events), int(gen_id), _ptr(p), _ptr(w), _ptr(st))
        if rc != OR_OK:
            raise RuntimeError(f"oracle generate failed ({rc})")
        nw = int(st[0])
        return {"p": p[:nw], "w": w[:nw], "n_written": nw, "n_calls_used": int(st[1]),
                "n_overweight": int(st[2]), "n_batches": int(st[3])}

    # -- state -------------------------------------------------------------
    def get_state(self):
        e = np.zeros((self.K, self.d, self.n + 1), np.float64)
        a = np.zeros(self.K, np.float64)
        s = np.zeros(self.K, np.float64)
        wm = C.c_double(0.0)
        self.lib.or_get_state(self.h, _ptr(e), _ptr(a), _ptr(s), C.byref(wm))
        return {"edges": e, "alpha": a, "shift": s, "w_max": wm.value}

    def set_state(self, edges=None, alpha=None, shift=None, w_max: float = 0.0,
                  have_pass: bool = True):
        e = None if edges is None else np.ascontiguousarray(edges, np.float64)
        a = None if alpha is None else np.ascontiguousarray(alpha, np.float64)
        s = None if shift is None else np.ascontiguousarray(shift, np.float64)
        self.lib.or_set_state(self.h, None if e is None else _ptr(e),
                              None if a is None else _ptr(a), None if s is None else _ptr(s),
                              float(w_max), int(bool(have_pass)))

    def get_pass(self):
        D = np.zeros((self.K, self.d, self.n), np.float64)
        Ic = np.zeros(self.K, np.float64)
        Vc = np.zeros(self.K, np.float64)
        Nc = np.zeros(self.K, np.int64)
        self.lib.or_get_pass(self.h, _ptr(D), _ptr(Ic), _ptr(Vc), _ptr(Nc))
        return {"D": D, "Ic": Ic, "Vc": Vc, "Nc": Nc}

    def get_pooled(self):
        """Bin weights the next refinement uses (after the equivalences, R18)."""
        D = np.zeros((self.K, self.d, self.n), np.float64)
        rc = self.lib.or_get_pooled(self.h, _ptr(D))
        if rc != OR_OK:
            raise RuntimeError(f"oracle get_pooled failed ({rc})")
        return D

    # -- point functions -----------------------------------------------------
    def f(self, p) -> float:
        p = np.ascontiguousarray(p, np.float64)
        return float(self.lib.or_f(self.h, _ptr(p)))

    def g(self, p) -> float:
        p = np.ascontiguousarray(p, np.float64)
        return float(self.lib.or_g_point(self.h, _ptr(p)))

    def grid_density(self, c: int, x) -> float:
        x = np.ascontiguousarray(x, np.float64)
        return float(self.lib.or_grid_density(self.h, int(c), _ptr(x)))

    def channel_forward(self, c: int, x):
        x = np.ascontiguousarray(x, np.float64)
        p = np.zeros(self.d, np.float64)
        j = C.c_double(0.0)
        self.lib.or_channel_forward(self.h, int(c), _ptr(x), _ptr(p), C.byref(j))
        return p, j.value

    def channel_inverse(self, c: int, p):
        p = np.ascontiguousarray(p, np.float64)
        x = np.zeros(self.d, np.float64)
        j = C.c_double(0.0)
        self.lib.or_channel_inverse(self.h, int(c), _ptr(p), _ptr(x), C.byref(j))
        return x, j.value

    def eval_call(self, mode: int, field: int, call: int, with_bins: bool = True):
        d, K = self.d, self.K
        x = np.zeros(d, np.float64)
        p = np.zeros(d, np.float64)
        jf = np.zeros(d, np.int32)
        bins = np.zeros(K * d, np.int32) if with_bins else None
        words = np.zeros(d + 2, np.uint32)
        o = np.zeros(4, np.float64)
        rc = self.lib.or_eval_call(self.h, int(mode), int(field), int(call), _ptr(x), _ptr(p),
                                   _ptr(jf), None if bins is None else _ptr(bins), _ptr(words),
                                   _ptr(o))
        if rc != OR_OK:
            raise RuntimeError(f"oracle eval_call failed ({rc})")
        return {"x": x, "p": p, "jf": jf, "bins": None if bins is None else bins.reshape(K, d),
                "words": words, "f": o[0], "g": o[1], "w": o[2], "channel": int(o[3])}

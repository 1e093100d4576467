"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point that include/vamp.h declares; host-side argument
validation rejects bad descriptors before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1811_09711_gb300 import build as B
from paper_1811_09711_gb300 import problems as P
from paper_1811_09711_gb300 import vamp as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(vamp_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return V.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_library_is_bound_to_its_sources(lib):
    """The loaded library carries the hash of the sources on disk, and the
    build script records the same hash beside it."""
    h = lib.vamp_source_hash().decode()
    assert len(h) == 64 and h == B.source_hash() == B.recorded_hash()


def test_status_strings_and_record_bytes(lib):
    assert lib.vamp_status_string(0) == b"VAMP_OK"
    assert lib.vamp_status_string(6) == b"VAMP_ERR_STATE"
    assert lib.vamp_status_string(7) == b"VAMP_ERR_LIMIT"
    assert lib.vamp_last_error(None) == b""
    assert [lib.vamp_record_bytes(d) for d in (1, 2, 3, 14, 16)] == [16, 16, 24, 64, 72]


def _create_status(lib, problem, **over):
    cfg, keep = V.make_config(problem)
    for k, v in over.items():
        setattr(cfg, k, v)
    h = C.c_void_p()
    return lib.vamp_create(C.byref(cfg), None, C.byref(h)), h


@pytest.mark.parametrize("field,value", [
    ("d", 0), ("d", 17), ("n_channels", 0), ("n_bins", 0), ("n_bins", 257), ("n_peaks", 0),
    ("grid_alpha", 0.0), ("n_min", 0), ("n_min", 1 << 32), ("gen_batch", -1), ("gen_batch", (1 << 24) + 1),
    ("precision", 2), ("gauss_sigma", -1.0),
])
def test_create_rejects_bad_config(lib, field, value):
    rc, h = _create_status(lib, P.bw_gauss(), **{field: value})
    assert rc == V.VAMP_ERR_INVALID_ARG and not h.value


def test_create_rejects_bad_maps(lib):
    pr = P.bw_gauss()
    bad = pr.channels.copy()
    bad.b[0, 0] = 0.0  # zero Breit-Wigner width
    assert _create_status(lib, pr.replace(channels=bad))[0] == V.VAMP_ERR_INVALID_ARG
    bad = pr.channels.copy()
    bad.n_mapped[1] = 2
    bad.coord[1, 1] = bad.coord[1, 0]  # coordinate mapped twice
    bad.kind[1, 1] = P.MAP_BW
    bad.b[1, 1] = 1e-3
    assert _create_status(lib, pr.replace(channels=bad))[0] == V.VAMP_ERR_INVALID_ARG
    bad = pr.peaks.copy()
    bad.coord[0, 0] = 8  # out of range for d = 8
    assert _create_status(lib, pr.replace(peaks=bad))[0] == V.VAMP_ERR_INVALID_ARG
    bad = pr.channels.copy()
    bad.kind[2, 0] = 7
    assert _create_status(lib, pr.replace(channels=bad))[0] == V.VAMP_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", ["stratified", "negative_count", "null_table", "channel", "partner",
                                 "axis", "not_perm", "kind"])
def test_create_rejects_bad_modes(lib, bad):
    """Pseudo-stratified flag and channel-equivalence tables are validated on
    the host, before any device work."""
    pr = P.ring(3, 6)
    if bad == "stratified":
        rc, h = _create_status(lib, pr, stratified=2)
    elif bad == "negative_count":
        rc, h = _create_status(lib, pr, n_equiv=-1)
    elif bad == "null_table":
        rc, h = _create_status(lib, pr.replace(equivalences=None), n_equiv=2)
    else:
        row = [0, 1] + list(range(6)) + [0] * 6
        if bad == "channel":
            row[0] = 3
        elif bad == "partner":
            row[1] = -1
        elif bad == "axis":
            row[2] = 6
        elif bad == "not_perm":
            row[3] = row[2]
        else:
            row[2 + 6] = 4
        rc, h = _create_status(lib, pr.replace(equivalences=np.array([row], np.int32)))
    assert rc == V.VAMP_ERR_INVALID_ARG and not h.value


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = _create_status(lib, P.bw_gauss())
    assert rc in (V.VAMP_ERR_CUDA, V.VAMP_ERR_OOM) and not h.value


def test_null_arguments(lib):
    h = C.c_void_p()
    assert lib.vamp_create(None, None, C.byref(h)) == V.VAMP_ERR_INVALID_ARG
    assert lib.vamp_sample_pass(None, 10, 0, None) == V.VAMP_ERR_INVALID_ARG
    assert lib.vamp_sample_pass_async(None, 10, 0, None) == V.VAMP_ERR_INVALID_ARG
    assert lib.vamp_refine_grids(None) == V.VAMP_ERR_INVALID_ARG
    lib.vamp_destroy(None)


def test_decode_records_layout():
    d = 3
    rb = 24
    raw = np.zeros(2 * rb, np.uint8)
    raw[:12] = np.frombuffer(np.array([1.5, 2.5, 3.5], np.float32).tobytes(), np.uint8)
    raw[16:24] = np.frombuffer(np.array([7.25]).tobytes(), np.uint8)
    p, w = V.decode_records(raw, d)
    assert p.shape == (2, 3) and list(p[0]) == [1.5, 2.5, 3.5] and w[0] == 7.25


def test_server_null_arguments(lib):
    h = C.c_void_p()
    assert lib.vamp_server_create(0, 1 << 30, 1, C.byref(h)) == V.VAMP_ERR_INVALID_ARG and not h.value
    assert lib.vamp_server_create(4, 0, 1, C.byref(h)) == V.VAMP_ERR_INVALID_ARG
    assert lib.vamp_server_create(4, 1 << 30, 2, C.byref(h)) == V.VAMP_ERR_INVALID_ARG
    cfg, keep = V.make_config(P.bw_gauss())
    rid = C.c_uint64()
    assert lib.vamp_server_submit(None, C.byref(cfg), 1, 100, 0, 0, None, C.byref(rid)) == V.VAMP_ERR_INVALID_ARG
    assert lib.vamp_server_poll(None, None, 4) == 0
    assert lib.vamp_server_wait_idle(None, 1.0) == V.VAMP_ERR_INVALID_ARG
    lib.vamp_server_destroy(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the C header's sizes and offsets
    (compiled with the host C compiler)."""
    structs = {
        "vamp_map_desc": V.MapDesc, "vamp_config": V.Config, "vamp_pass_result": V.PassResult,
        "vamp_request_result": V.RequestResult,
    }
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vamp.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_selftest_bounded_wait_rejects_bad_limits(lib):
    import ctypes as C
    cyc = C.c_int64()
    assert lib.vamp_selftest_bounded_wait(0, C.byref(cyc)) == V.VAMP_ERR_INVALID_ARG
    assert lib.vamp_selftest_bounded_wait((1 << 31) + 1, C.byref(cyc)) == V.VAMP_ERR_INVALID_ARG

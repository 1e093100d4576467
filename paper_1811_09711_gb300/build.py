"""In-tree build of the CUDA library (sm_103a) with nvcc.

Produces ``paper_1811_09711_gb300/_lib/libvamp_gb300.so`` from the sources
in ``csrc/``; translation units compile in parallel, then link once.

The library is bound to the sources it was built from: a SHA-256 over every
source and header and the compiler flags is compiled into it
(``vamp_source_hash()``) and written beside it.  ``build()`` recompiles
whenever the recorded hash differs from the hash of the sources on disk
(not by file times), and the binding refuses a library whose embedded hash
does not match the sources, so a run always executes the committed code.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libvamp_gb300.so")
HASH_FILE = os.path.join(LIBDIR, "libvamp_gb300.sha256")
SOURCES = ["vamp_api.cu", "vamp_setup.cu", "vamp_kernels.cu", "vamp_noalloc.cu", "vamp_pass_f32.cu",
           "vamp_pass_f32_shapes.cu", "vamp_pass_f64.cu", "vamp_batch.cu", "vamp_batch_pass.cu",
           "vamp_server.cu", "vamp_peaks.cu", "vamp_union.cu"]
HEADERS = ["vamp_device.cuh", "vamp_internal.h", "vamp_pass.cuh", "vamp_union.cuh",
           os.path.join("..", "..", "include", "vamp.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def source_hash() -> str:
    """SHA-256 of the sources, headers, flags and this build script."""
    h = hashlib.sha256()
    for name in sorted(SOURCES + HEADERS) + [os.path.abspath(__file__)]:
        path = name if os.path.isabs(name) else os.path.join(CSRC, name)
        h.update(os.path.basename(path).encode() + b"\0")
        with open(path, "rb") as f:
            h.update(f.read())
        h.update(b"\0")
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def recorded_hash() -> str | None:
    """Hash recorded beside the built library, None if there is none."""
    if not (os.path.exists(LIB) and os.path.exists(HASH_FILE)):
        return None
    with open(HASH_FILE) as f:
        return f.read().strip() or None


def _stale() -> bool:
    return recorded_hash() != source_hash()


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    digest = source_hash()
    objs = []

    def compile_one(src):
        obj = os.path.join(LIBDIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, f"-DVAMP_SOURCE_HASH=\"{digest}\"", "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        for obj, log in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if verbose and log:
                print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    if os.path.exists(HASH_FILE):
        os.remove(HASH_FILE)
    os.replace(tmp, LIB)
    with open(HASH_FILE + f".tmp{os.getpid()}", "w") as f:
        f.write(digest + "\n")
    os.replace(HASH_FILE + f".tmp{os.getpid()}", HASH_FILE)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))

"""Build libvcs.so (the CUDA hot path and its C ABI) for sm_103a, in-tree."""
from __future__ import annotations

import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libvcs.so")
SOURCES = ["vcs_kernels.cu", "vcs_kernels_xm.cu", "vcs_kernels_ft.cu", "vcs_soft.cu", "vcs_api.cu", "vcs_full.cu",
           "vcs_raster.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2"]


OBJ_DIR = os.path.join(HERE, "_build")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(HERE, "..", "include", "vcs.h"), os.path.abspath(__file__)]


def _obj(src: str) -> str:
    return os.path.join(OBJ_DIR, src.replace(".cu", ".o"))


def _deps(path: str, seen=None) -> set:
    """The file and every file it includes with #include "..." (recursively)."""
    seen = set() if seen is None else seen
    path = os.path.normpath(path)
    if path in seen or not os.path.exists(path):
        return seen
    seen.add(path)
    for ln in open(path):
        m = re.match(r'\s*#\s*include\s+"([^"]+)"', ln)
        if m:
            _deps(os.path.join(os.path.dirname(path), m.group(1)), seen)
    return seen


def _stale_sources(force: bool):
    """Sources whose object is missing or older than the source or a header
    it includes (a change of FLAGS needs build(force=True))."""
    out = []
    for src in SOURCES:
        o = _obj(src)
        deps = _deps(os.path.join(CSRC, src))
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(f) for f in deps):
            out.append(src)
    return out


def stale() -> bool:
    """The library is missing or older than a source or header (the objects
    need not be present: a copy of the tree with a current library is
    current)."""
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _headers() + [os.path.join(CSRC, s) for s in SOURCES])


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (those whose inputs changed; the
    objects are kept under _build/) and link libvcs.so."""
    if not force and not stale():
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)

    def compile_one(src):
        tmp = _obj(src) + f".tmp{os.getpid()}"
        cmd = [NVCC, *FLAGS, "-c", os.path.join(CSRC, src), "-o", tmp]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
        os.replace(tmp, _obj(src))

    todo = _stale_sources(force)
    if todo:
        with ThreadPoolExecutor(len(todo)) as ex:
            list(ex.map(compile_one, todo))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "-shared", *[_obj(s) for s in SOURCES], "-o", tmp, "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="-f" in sys.argv, verbose="-v" in sys.argv))

"""Build libdgconv.so in-tree for sm_103a (GB300), and its checked twin.

The C++ table builder is compiled by g++, the CUDA sources by nvcc with
``-gencode arch=compute_103a,code=sm_103a``; translation units compile in
parallel and are linked against the shared CUDA runtime.  The same sources
compiled with ``-DDGC_CHECKED=1`` give libdgconv_checked.so, whose kernels
bounds-check every gather index (a test build; the binding loads it when
DGC_LIBRARY=checked).  Rebuilds only when a source is newer than a library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdgconv.so")
LIB_CHECKED = os.path.join(PKG, "libdgconv_checked.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(src: str, extra=(), outdir: str = BUILD) -> str:
    obj = os.path.join(outdir, os.path.basename(src) + ".o")
    if src.endswith(".cpp"):
        cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-I", INCLUDE, *extra, "-c", src, "-o", obj]
    else:
        cmd = [_nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    return obj


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def _link(objs, lib: str) -> None:
    tmp = lib + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    """Both libraries (the regular and the checked one); returns the regular one's path."""
    jobs = []
    if force or _stale(LIB):
        os.makedirs(BUILD, exist_ok=True)
        jobs += [(src, (), BUILD, LIB) for src in _sources()]
    if force or _stale(LIB_CHECKED):
        os.makedirs(BUILD_CHECKED, exist_ok=True)
        jobs += [(src, ("-DDGC_CHECKED=1",), BUILD_CHECKED, LIB_CHECKED) for src in _sources()]
    if not jobs:
        return LIB
    with cf.ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(lambda j: (j[3], _compile(j[0], j[1], j[2])), jobs))
    for lib in (LIB, LIB_CHECKED):
        mine = [o for l, o in objs if l == lib]
        if mine:
            _link(mine, lib)
            if verbose:
                print("built", lib)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)

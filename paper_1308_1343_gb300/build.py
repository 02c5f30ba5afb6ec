"""Build libsc_level.so in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel into ``_build/`` and linked
into ``paper_1308_1343_gb300/libsc_level.so``.  A build is skipped when the
library is newer than every source and header.

``build(checked=True)`` makes ``libsc_level_checked.so`` instead: the same
sources with ``SC_BOUNDS_CHECK`` defined, whose traversal verifies every
element index against its box and reports a failure through the error word
(a stand-in for a device memory checker).  Point the Python binding at it
with the environment variable ``SC_LEVEL_LIB``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsc_level.so")
LIB_CHECKED = os.path.join(HERE, "libsc_level_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kernels.cu", "runtime.cu", "autotune.cu", "noalloc.cu", "hierarchy.cu",
           "level_host.cpp"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += glob.glob(os.path.join(CSRC, "*.hpp")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    files += glob.glob(os.path.join(ROOT, "include", "*.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(src: str, verbose_ptxas: bool, checked: bool = False) -> str:
    out = os.path.join(BUILD, "checked") if checked else BUILD
    obj = os.path.join(out, os.path.basename(src) + ".o")
    cmd = [_nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    if checked:
        cmd.insert(1, "-DSC_BOUNDS_CHECK")
    if verbose_ptxas and src.endswith(".cu"):
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    """Compile and link the library (or its checked build); returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib):
        return lib
    os.makedirs(os.path.join(BUILD, "checked") if checked else BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas, checked), SOURCES))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt",
           "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                checked="--checked" in sys.argv))

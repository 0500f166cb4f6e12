"""Build the GB300 GMRES library (libgmres_gb300.so) in-tree with nvcc.

The CUDA sources under csrc/ are compiled for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), in parallel, into a shared
library next to this file.  No CMake, no torch extension machinery: the
library exposes a plain C ABI (include/gmres_gb300.h) that the ctypes binding
in gmres.py loads.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libgmres_gb300.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)
BUILD_DIR = os.path.join(ROOT, "_build")
# the checked build: the same sources with -DGMRES_CHECKS (column indices
# tested in every gather kernel; include/gmres_gb300.h, gmres_checks_enabled)
LIB_CHECKED_PATH = os.path.join(HERE, "libgmres_gb300_checked.so")
BUILD_DIR_CHECKED = os.path.join(ROOT, "_build", "checked")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xptxas", "-O3"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _units():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files


def stale(checked: bool = False) -> bool:
    path = LIB_CHECKED_PATH if checked else LIB_PATH
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile every .cu under csrc/ and link libgmres_gb300.so (if stale);
    with checked=True the checked build libgmres_gb300_checked.so instead."""
    lib_path = LIB_CHECKED_PATH if checked else LIB_PATH
    build_dir = BUILD_DIR_CHECKED if checked else BUILD_DIR
    if checked:
        extra = (*extra, "-DGMRES_CHECKS")
    if not force and not stale(checked):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    nv = nvcc()
    units = _units()

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        cmd = [nv, *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = lib_path + ".tmp%d" % os.getpid()
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


def build_all(force: bool = False, verbose: bool = False):
    """Both libraries, the normal and the checked build, compiled side by side
    (their units share one machine's cores); returns the two paths."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        normal = ex.submit(build, force, verbose)
        checked = ex.submit(build, force, verbose, (), True)
        return normal.result(), checked.result()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))

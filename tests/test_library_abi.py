"""The compiled library loads and exports every symbol the C header declares.

CPU-only (no compute call needs a GPU): the library is built with nvcc for
sm_103a, loaded with ctypes, and each ``extern "C"`` declaration found in
include/*.h is looked up.  Also checks that the Python binding's signature
table covers exactly the declared entry points.
"""
import ctypes
import os
import re

import pytest

from paper_2011_01850_gb300 import build as B
from paper_2011_01850_gb300 import gmres as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(gmres_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def so():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("gmres_create", "gmres_solve", "gmres_destroy", "gmres_spmv",
                 "gmres_residual", "gmres_arnoldi", "gmres_status_str"):
        assert must in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in sorted(declared_functions()) if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(G.SIGNATURES) == declared_functions()


def test_checked_build_exports_and_reports(so):
    """The checked build (-DGMRES_CHECKS) exports the same entry points and
    says it is the checked build; the normal build says it is not."""
    L = ctypes.CDLL(B.build(checked=True))
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing
    for lib_, want in ((L, 1), (so, 0)):
        lib_.gmres_checks_enabled.restype = ctypes.c_int32
        lib_.gmres_checks_enabled.argtypes = []
        assert lib_.gmres_checks_enabled() == want


def test_host_only_calls(so):
    # calls that touch no device: status strings, version, default options
    G._lib = None
    assert G.gmres_status_str(G.OK) == "converged"
    assert G.gmres_status_str(G.ERR_ARG) == "invalid argument"
    assert "checked build" in G.gmres_status_str(G.ERR_INDEX)
    assert "sm_103a" in G.gmres_version()
    o = G.gmres_default_opts()
    assert o.tau < 0 and o.inner_factor == 0.5 and o.repeat_first == -1


def test_built_for_sm103a_only():
    # the build passes exactly one -gencode, for sm_103a
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_header_is_plain_c_and_links_from_c(so, tmp_path):
    """The C-ABI is usable from C: the header compiles as C99 with warnings
    as errors, and a C program linked against the library calls its
    host-only entry points (status strings, default options, version)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = tmp_path / "use_abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "gmres_gb300.h"
int main(void) {
    gmres_opts o;
    gmres_default_opts(&o);
    if (o.inner_factor != 0.5 || o.repeat_first != -1 || o.trsv_kernel != 0) return 2;
    if (strcmp(gmres_status_str(GMRES_OK), "converged") != 0) return 3;
    if (strstr(gmres_version(), "sm_103a") == NULL) return 4;
    printf("%s\n", gmres_status_str(GMRES_ERR_ARG));
    return 0;
}
''')
    lib = B.build()
    exe = tmp_path / "use_abi"
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           lib, "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.strip() == "invalid argument"


def test_no_library_no_fallback(monkeypatch, tmp_path):
    """Without the compiled library every entry point raises: there is no
    CPU fallback behind the binding."""
    monkeypatch.setattr(G, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(G, "_lib", None)
    with pytest.raises(RuntimeError, match="no fallback"):
        G.lib()
    import numpy as np
    A = (np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.0]))
    with pytest.raises(RuntimeError, match="no fallback"):
        G.Solver(A)

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


def test_host_only_calls(so):
    # calls that touch no device: status strings, version, default options
    G._lib = None
    assert G.gmres_status_str(G.OK) == "converged"
    assert G.gmres_status_str(G.ERR_ARG) == "invalid argument"
    assert "sm_103a" in G.gmres_version()
    o = G.gmres_default_opts()
    assert o.tau < 0 and o.inner_factor == 0.5 and o.repeat_first == -1


def test_built_for_sm103a_only():
    # the build passes exactly one -gencode, for sm_103a
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]

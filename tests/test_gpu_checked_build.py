"""The checked build (-DGMRES_CHECKS) on the GPU (marker: gpu).

The checked build tests every column index a kernel gathers x with against
its system's columns, counts an index outside, and replaces it by column 0
so the load stays in bounds; the entry points then return GMRES_ERR_INDEX.
Run in a child process with GMRES_GB300_CHECKS=1 (the binding loads one
library per process):

* valid systems give no false report: the no-allocation solve, a grid-path
  solve with A's sliced copy and the products in both storages succeed, with
  the oracle's residual;
* one planted column index n (one past the last column) in the matrix given
  to gmres_solve_noalloc, the entry point that does not validate columns on
  the host, is reported as GMRES_ERR_INDEX in binary64 and binary32;
* the next valid call is clean again (the check word is cleared).

The planted index reads, were a path left unchecked, one entry past x: the
system has 1023 rows, the basis columns are padded to 1024 and x's device
allocation to a multiple of 512 bytes, so even then no load leaves an
allocation.
"""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r'''
    import sys
    sys.path.insert(0, %r)
    import numpy as np
    import torch
    import oracle as O
    from paper_2011_01850_gb300 import build as B
    B.build(checked=True)
    from paper_2011_01850_gb300 import gmres as G
    from paper_2011_01850_gb300 import inputs as I

    assert G.CHECKED and G.gmres_checks_enabled() == 1
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    A = I.convdiff2d(33, 31, pe=10.0)                  # n = 1023
    rp, ci, va = A
    n, nnz = len(rp) - 1, len(ci)
    b = I.rhs_ones_noise(A, 1e-3, 5)
    dev = lambda a, dt: torch.tensor(np.asarray(a), dtype=dt, device="cuda")
    drp, dva, db = dev(rp, torch.int32), dev(va, torch.float64), dev(b, torch.float64)

    def noalloc(cols, prec):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        try:
            st, info = G.gmres_solve_noalloc(n, drp, cols, dva, nnz, db, x, 30, 1e-10,
                                             G.ORTHO_CGSR, prec, 300, stream)
        except G.GmresError as e:
            return e.status, None
        return st, x.cpu().numpy()

    good = dev(ci, torch.int32)
    bad_ci = np.array(ci, np.int32)
    bad_ci[nnz // 2] = n                                # one column past the end
    bad = dev(bad_ci, torch.int32)
    for prec in (G.FP64, G.MIXED):
        st, x = noalloc(good, prec)
        assert st == G.OK, ("valid system reported", prec, st)
        assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
        st, _ = noalloc(bad, prec)
        assert st == G.ERR_INDEX, ("planted column not reported", prec, st)
        st, x = noalloc(good, prec)                     # the word was cleared
        assert st == G.OK, ("report leaked into the next call", prec, st)

    # handle paths on a validated matrix: no false reports
    s = G.Solver(A, stream=stream)
    s.set_opts(spmv_format=G.SPMV_SLICED, path=G.PATH_GRID)
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, st, info = s.solve(db, dx, m=30, tol=1e-10, ortho="cgsr", prec="mixed")
    assert st == G.OK, st
    assert O.residual_norm(A, b, dx.cpu().numpy()) / np.linalg.norm(b) <= 1e-10
    xv = np.random.default_rng(1).standard_normal(n)
    for fmt in (G.SPMV_CSR, G.SPMV_SLICED):
        s.set_opts(spmv_format=fmt)
        y = torch.zeros(n, dtype=torch.float64, device="cuda")
        G.gmres_spmv(s.h, dev(xv, torch.float64), y, G.FP64)
        yo = O.spmv(A, xv, O.FP64)
        assert np.abs(y.cpu().numpy() - yo).max() <= 1e-13 * np.abs(yo).max()
    s.close()
    print("CHECKED-BUILD-OK")
''') % ROOT


def test_checked_build_reports_bad_columns(gpulib):
    env = dict(os.environ, GMRES_GB300_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "CHECKED-BUILD-OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]

"""The benchmarked configuration at full size (marker: gpu).

160^3 convection-diffusion (n = 4 096 000, nnz = 28 518 400), mixed CGSR
GMRES(100) in the launch configuration bench.py times (autotuned SpMV lanes,
grid path).  The oracle cannot solve this size in test time, so the checks are
the ones that hold at any size: the binary64 relative residual of the returned
x, recomputed by the oracle, is <= 1e-10; the mixed solve reaches the same
residual class as the binary64 solve; and the SpMV kernels match the oracle on
sampled rows (full binary64/binary32 oracle SpMV, rows sampled for the
element-wise gamma_k comparison).
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G


@pytest.fixture(scope="module")
def full():
    A, b, spec = I.workload("convdiff3d_160", seed=20110185)
    return A, b, spec


def test_fullsize_spmv_sampled_rows(full, gpulib):
    A, b, spec = full
    rp, ci, va = A
    n = len(rp) - 1
    s = G.Solver(A, stream=torch.cuda.current_stream())
    G.gmres_autotune(s.h)
    x = np.random.default_rng(1).standard_normal(n)
    rows = np.random.default_rng(2).choice(n, 4096, replace=False)
    k = np.diff(rp)[rows].astype(np.float64)
    for prec, dt, u in ((G.FP64, torch.float64, 2.0 ** -53), (G.MIXED, torch.float32, 2.0 ** -24)):
        y = torch.zeros(n, dtype=dt, device="cuda")
        G.gmres_spmv(s.h, torch.tensor(x, dtype=dt, device="cuda"), y, prec)
        yo = O.spmv(A, x, O.FP64 if prec == G.FP64 else O.MIXED)
        xs = x.astype(np.float32).astype(np.float64) if prec else x
        ab = np.array([np.sum(np.abs(va[rp[r]:rp[r + 1]]) * np.abs(xs[ci[rp[r]:rp[r + 1]]]))
                       for r in rows])
        g = k * u / (1 - k * u)
        assert np.all(np.abs(y.cpu().numpy()[rows] - yo[rows]) <= 2 * g * ab * 1.0001 + 1e-300)
    s.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_fullsize_solve_residual(full, prec, gpulib):
    A, b, spec = full
    n = len(A[0]) - 1
    s = G.Solver(A, stream=torch.cuda.current_stream())
    G.gmres_autotune(s.h)
    db = torch.tensor(b, device="cuda", dtype=torch.float64)
    dx = torch.zeros(n, device="cuda", dtype=torch.float64)
    _, st, info = s.solve(db, dx, m=spec["m"], tol=1e-10, ortho=spec["ortho"], prec=prec,
                          maxiter=100000)
    s.close()
    assert st == G.OK, info
    assert info["path"] == G.PATH_GRID
    x = dx.cpu().numpy()
    rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
    assert rel <= 1e-10, rel
    assert abs(rel - info["relres"]) <= 1e-6 * rel
    # the solution of b = A 1 + noise is close to 1 (noise 1e-3 per entry)
    assert np.abs(x - 1.0).max() < 0.5

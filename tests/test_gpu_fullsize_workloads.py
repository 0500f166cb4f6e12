"""Two more benchmarked workloads at full size (marker: gpu).

* ILU(0) on the 160^3 convection-diffusion matrix (n = 4 096 000,
  nnz = 28 518 400): the factors and the binary64 preconditioner apply
  (L then U, with the kernels chosen as in a solve) equal the oracle's bit for
  bit on every row, and the preconditioned mixed CGSR GMRES(100) solve reaches
  a binary64 relative residual <= 1e-10 (recomputed by the oracle) in fewer
  iterations than the unpreconditioned one.
* The 2048-system batch (sizes log-uniform in [500, 50000], seed of the
  benchmark's first rank): every system's solution has an oracle-recomputed
  relative residual <= 1e-10, and the residual each system reports agrees.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G

SEED = 20110185


@pytest.fixture(scope="module")
def ilu160():
    A, b, spec = I.workload("convdiff3d_160_ilu", seed=SEED)
    return A, b, spec, O.ilu0(A)


def test_fullsize_ilu_factors_and_apply_bitwise(ilu160, gpulib):
    A, b, spec, LU = ilu160
    n = len(b)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    G.gmres_ilu0(s.h)
    assert G.gmres_ilu_levels(s.h) == (478, 478)  # 3N - 2 for N = 160
    assert np.array_equal(G.gmres_ilu_factors(s.h, len(A[1])), LU[2])
    z = np.random.default_rng(3).standard_normal(n)
    want = O.ilu_apply(LU, z)
    out = torch.zeros(n, device="cuda", dtype=torch.float64)
    G.gmres_ilu_apply(s.h, torch.tensor(z, device="cuda"), out, G.FP64)
    s.close()
    assert np.array_equal(out.cpu().numpy(), want)


def test_fullsize_ilu_solve(ilu160, gpulib):
    A, b, spec, _ = ilu160
    n = len(b)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    G.gmres_autotune(s.h)
    G.gmres_ilu0(s.h)
    s.set_opts(precond=G.PRECOND_ILU0)
    db = torch.tensor(b, device="cuda", dtype=torch.float64)
    dx = torch.zeros(n, device="cuda", dtype=torch.float64)
    _, st, info = s.solve(db, dx, m=spec["m"], tol=1e-10, ortho=spec["ortho"], prec=spec["prec"],
                          maxiter=100000)
    s.close()
    assert st == G.OK, info
    x = dx.cpu().numpy()
    rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
    assert rel <= 1e-10, rel
    # the unpreconditioned solve of this system takes 1300 inner iterations
    assert info["iters"] < 600, info


def test_fullsize_batched_2048(gpulib):
    systems = I.batched_convdiff2d(count=2048, nmin=500, nmax=50000, seed=SEED)
    sys_ptr, rp, ci, va, b = G.pack_batch(systems)
    nsys = len(systems)
    h = G.gmres_batch_create(nsys, sys_ptr, rp, ci, va, stream=torch.cuda.current_stream())
    db = torch.tensor(b, device="cuda", dtype=torch.float64)
    dx = torch.zeros(len(b), device="cuda", dtype=torch.float64)
    st, res, info = G.gmres_batch_solve(h, db, dx, 30, 1e-10, G.ORTHO_MGS, G.MIXED, 100000,
                                        nsys=nsys)
    G.gmres_batch_destroy(h)
    assert st == G.OK and info.converged == 1
    x = dx.cpu().numpy()
    for i, (A, bi) in enumerate(systems):
        xi = x[sys_ptr[i]:sys_ptr[i + 1]]
        rel = O.residual_norm(A, bi, xi) / np.linalg.norm(bi)
        assert rel <= 1e-10, (i, rel)
        assert res[i].converged == 1 and abs(res[i].relres - rel) <= 1e-3 * rel + 1e-14, i

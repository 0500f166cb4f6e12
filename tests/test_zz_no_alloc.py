"""gmres_solve_noalloc, the entry point for callers that cannot allocate
device memory at solve time (marker: gpu).

It must give the same solution as the allocating entry point gmres_solve on
the same path (the single-block solver), on two calls in a row -- the second
call finds the shared scratch array holding the first call's data -- and it
must reject a system whose workspace exceeds the scratch.  This file runs
last so that a failure here comes after every other test has run; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G


def _dev(a, dt):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("prec,ortho,N", [("mixed", "mgs", 40), ("fp64", "cgsr", 40),
                                           ("mixed_bf16", "cgsr", 40), ("fp64", "mgs", 48)])
def test_noalloc_matches_allocating_solve(prec, ortho, N, gpulib):
    A = I.convdiff2d(N, pe=10.0)           # n = 1600, and 2304 (binary64: one block here)
    rp, ci, va = A
    n, nnz = len(rp) - 1, len(ci)
    b = I.rhs_ones_noise(A, 1e-3, 3)
    stream = torch.cuda.current_stream()
    # the existing entry point, same path (one thread block per system)
    s = G.Solver(A, stream=stream)
    s.set_opts(path=G.PATH_BLOCK, block_cluster=1)
    xr = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, st_ref, info_ref = s.solve(_dev(b, torch.float64), xr, m=30, tol=1e-10, ortho=ortho,
                                  prec=prec, maxiter=4000)
    s.close()
    assert st_ref == G.OK
    xr = xr.cpu().numpy()
    drp, dci, dva = _dev(rp, torch.int32), _dev(ci, torch.int32), _dev(va, torch.float64)
    db = _dev(b, torch.float64)
    for call in range(2):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = G.gmres_solve_noalloc(n, drp, dci, dva, nnz, db, x, 30, 1e-10,
                                         G.ORTHOS[ortho], G.PRECISIONS[prec], 4000, stream)
        assert st == G.OK, (call, st)
        x = x.cpu().numpy()
        # same kernel, same data: within the tolerance of the parity tests
        assert np.abs(x - xr).max() <= 1e-12 * np.abs(xr).max(), call
        assert info.iters == info_ref["iters"] and info.restarts == info_ref["restarts"]
        assert info.relres <= 1e-10
        # the binary64 residual of the returned x, recomputed by the oracle
        rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
        assert rel <= 1e-10, (call, rel)
        assert abs(rel - info.relres) <= 1e-6 * rel + 1e-15


def test_noalloc_rejects_inconsistent_nnz(gpulib):
    A = I.convdiff2d(20, pe=10.0)
    rp, ci, va = A
    n, nnz = len(rp) - 1, len(ci)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GmresError) as e:
        G.gmres_solve_noalloc(n, _dev(rp, torch.int32), _dev(ci, torch.int32),
                              _dev(va, torch.float64), nnz - 5, _dev(np.ones(n), torch.float64),
                              x, 30, 1e-10, G.ORTHO_MGS, G.MIXED, 100,
                              torch.cuda.current_stream())
    assert e.value.status == G.ERR_ARG


def test_noalloc_rejects_oversized_system(gpulib):
    A = I.convdiff2d(400, pe=10.0)         # n = 160000: (m+1) n s_V is far above 32 MiB
    rp, ci, va = A
    n, nnz = len(rp) - 1, len(ci)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GmresError) as e:
        G.gmres_solve_noalloc(n, _dev(rp, torch.int32), _dev(ci, torch.int32),
                              _dev(va, torch.float64), nnz, _dev(np.ones(n), torch.float64), x,
                              100, 1e-10, G.ORTHO_MGS, G.FP64, 100,
                              torch.cuda.current_stream())
    assert e.value.status == G.ERR_ARG

"""Batched solver against the oracle, system by system (marker: gpu).

Uneven 2-D convection-diffusion systems (sizes log-uniform, per-system
Peclet numbers) and power-law systems in one block-diagonal batch, solved in
one persistent launch; every system must reach a binary64 relative residual
<= 1e-10 (recomputed by the oracle) and match the oracle's solution.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G


def _systems():
    sys = I.batched_convdiff2d(count=24, nmin=40, nmax=3000, seed=5)
    sys += [(I.powerlaw_random(n, seed=n), None) for n in (50, 777)]
    sys += [(I.dense_to_csr(np.array([[3.0]])), None)]
    out = []
    for k, (A, b) in enumerate(sys):
        if b is None:
            b = I.rhs_ones_noise(A, 1e-3, 100 + k)
        out.append((A, b))
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16", "mixed_fp16"])
@pytest.mark.parametrize("ortho", ["mgs", "cgsr"])
def test_batch_parity(prec, ortho, gpulib):
    systems = _systems()
    sys_ptr, rp, ci, va, b = G.pack_batch(systems)
    nsys = len(systems)
    h = G.gmres_batch_create(nsys, sys_ptr, rp, ci, va)
    x = np.zeros(len(b))
    st, res, info = G.gmres_batch_solve(h, b, x, 30, 1e-10, G.ORTHOS[ortho],
                                        G.PRECISIONS[prec], 4000, nsys=nsys)
    G.gmres_batch_destroy(h)
    assert st == G.OK, [(r.status, r.relres) for r in res]
    assert info.converged == 1
    for i, (A, bi) in enumerate(systems):
        xi = x[sys_ptr[i]:sys_ptr[i + 1]]
        rel = O.residual_norm(A, bi, xi) / np.linalg.norm(bi)
        assert rel <= 1e-10, (i, rel)
        assert res[i].converged == 1 and abs(res[i].relres - rel) <= 1e-3 * rel + 1e-14
        xo, _ = O.gmres(A, bi, m=30, tol=1e-13, ortho=O.CGSR, prec=O.FP64, maxiter=20000)
        kappa = np.linalg.cond(I.csr_to_dense(A)) if len(bi) <= 800 else 1e3
        err = np.linalg.norm(xi - xo) / np.linalg.norm(xo)
        assert err <= max(1e-8, 2 * kappa * (rel + 1e-13)), (i, err)


def test_batch_matches_single_solves_fp64(gpulib):
    """Binary64: a system solved inside the batch takes the same restart
    schedule as the same system solved alone (block path)."""
    systems = _systems()[:6]
    sys_ptr, rp, ci, va, b = G.pack_batch(systems)
    h = G.gmres_batch_create(len(systems), sys_ptr, rp, ci, va)
    x = np.zeros(len(b))
    st, res, info = G.gmres_batch_solve(h, b, x, 20, 1e-10, G.ORTHO_MGS, G.FP64, 4000,
                                        nsys=len(systems))
    G.gmres_batch_destroy(h)
    for i, (A, bi) in enumerate(systems):
        s = G.Solver(A)
        s.set_opts(path=G.PATH_BLOCK)
        xs, st1, inf1 = s.solve(bi, np.zeros(len(bi)), m=20, ortho="mgs", prec="fp64")
        s.close()
        assert inf1["iters"] == res[i].iters and inf1["restarts"] == res[i].restarts


def test_batch_rejects_cross_system_columns(gpulib):
    systems = _systems()[:3]
    sys_ptr, rp, ci, va, b = G.pack_batch(systems)
    ci = ci.copy()
    ci[0] = sys_ptr[2]  # a column of system 2 inside system 0
    with pytest.raises(G.GmresError) as e:
        G.gmres_batch_create(3, sys_ptr, rp, ci, va)
    assert e.value.status == G.ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_fp16"])
@pytest.mark.parametrize("ortho", ["mgs", "cgsr"])
def test_batch_cluster_path(prec, ortho, gpulib):
    """Systems of >= 8192 rows go to thread-block clusters (reductions over
    distributed shared memory) while the small ones run one block each, in
    a concurrent launch; both kinds must converge and match the oracle."""
    systems = [(I.convdiff2d(130, 130, pe=20.0), None), (I.convdiff2d(128, 160, pe=5.0), None)]
    systems += I.batched_convdiff2d(count=5, nmin=40, nmax=2000, seed=11)
    out = []
    for k, (A, b) in enumerate(systems):
        out.append((A, I.rhs_ones_noise(A, 1e-3, 300 + k) if b is None else b))
    sys_ptr, rp, ci, va, b = G.pack_batch(out)
    nsys = len(out)
    h = G.gmres_batch_create(nsys, sys_ptr, rp, ci, va)
    x = np.zeros(len(b))
    st, res, info = G.gmres_batch_solve(h, b, x, 30, 1e-10, G.ORTHOS[ortho],
                                        G.PRECISIONS[prec], 20000, nsys=nsys)
    G.gmres_batch_destroy(h)
    assert st == G.OK, [(r.status, r.relres) for r in res]
    assert info.kernel_launches[G.K_BLOCK] == 2
    for i, (A, bi) in enumerate(out):
        xi = x[sys_ptr[i]:sys_ptr[i + 1]]
        rel = O.residual_norm(A, bi, xi) / np.linalg.norm(bi)
        assert rel <= 1e-10, (i, rel)
        assert res[i].converged == 1 and abs(res[i].relres - rel) <= 1e-3 * rel + 1e-14
        xo, _ = O.gmres(A, bi, m=30, tol=1e-13, ortho=O.CGSR, prec=O.FP64, maxiter=40000)
        err = np.linalg.norm(xi - xo) / np.linalg.norm(xo)
        assert err <= 1e-6, (i, err)


def test_batch_autotune(gpulib):
    """The SpMV lanes autotuner picks a power of two in [1, 16], leaves the
    batch's x alone, and a later solve with lanes = 0 uses the choice and
    converges like an explicit one."""
    systems = _systems()
    sys_ptr, rp, ci, va, b = G.pack_batch(systems)
    nsys = len(systems)
    h = G.gmres_batch_create(nsys, sys_ptr, rp, ci, va)
    L = G.gmres_batch_autotune(h, b, 30, G.ORTHO_MGS, G.MIXED, 40)
    assert L in (1, 2, 4, 8, 16)
    x0 = np.zeros(len(b))
    st0, r0, _ = G.gmres_batch_solve(h, b, x0, 30, 1e-10, G.ORTHO_MGS, G.MIXED, 4000, nsys=nsys)
    x1 = np.zeros(len(b))
    st1, r1, _ = G.gmres_batch_solve(h, b, x1, 30, 1e-10, G.ORTHO_MGS, G.MIXED, 4000, lanes=L,
                                     nsys=nsys)
    G.gmres_batch_destroy(h)
    assert st0 == st1 == G.OK
    assert np.array_equal(x0, x1)
    assert [r.iters for r in r0] == [r.iters for r in r1]


def test_batch_cluster_threshold(gpulib):
    """Moving the cluster threshold moves systems between the one-block and
    the cluster launch; the results stay converged either way."""
    systems = [(I.convdiff2d(130, 130, pe=20.0), None)]
    systems += I.batched_convdiff2d(count=3, nmin=40, nmax=2000, seed=12)
    out = [(A, I.rhs_ones_noise(A, 1e-3, 400 + k) if b is None else b)
           for k, (A, b) in enumerate(systems)]
    sys_ptr, rp, ci, va, b = G.pack_batch(out)
    h = G.gmres_batch_create(len(out), sys_ptr, rp, ci, va)
    for rows, launches in ((0, 1), (1, 1), (16384, 2)):
        G.gmres_batch_set_cluster_rows(h, rows)
        x = np.zeros(len(b))
        st, res, info = G.gmres_batch_solve(h, b, x, 30, 1e-10, G.ORTHO_MGS, G.MIXED, 20000,
                                            nsys=len(out))
        assert st == G.OK and info.kernel_launches[G.K_BLOCK] == launches, rows
        for i, (A, bi) in enumerate(out):
            xi = x[sys_ptr[i]:sys_ptr[i + 1]]
            assert O.residual_norm(A, bi, xi) / np.linalg.norm(bi) <= 1e-10
    with pytest.raises(G.GmresError):
        G.gmres_batch_set_cluster_rows(h, -1)
    G.gmres_batch_destroy(h)


@pytest.mark.parametrize("threads", [128, 512, 1024])
def test_batch_cluster_threads(threads, gpulib):
    """The large systems' clusters run with any block size the setting
    allows (the rows are split over more or fewer threads); every system
    still converges to the binary64 target, in a number of iterations close
    to the oracle's."""
    systems = [(I.convdiff2d(110, 97, pe=30.0), None), (I.convdiff2d(90, 120, pe=5.0), None)]
    systems += I.batched_convdiff2d(count=4, nmin=100, nmax=3000, seed=13)
    out = [(A, I.rhs_ones_noise(A, 1e-3, 500 + k) if b is None else b)
           for k, (A, b) in enumerate(systems)]
    sys_ptr, rp, ci, va, b = G.pack_batch(out)
    h = G.gmres_batch_create(len(out), sys_ptr, rp, ci, va)
    G.gmres_batch_set_cluster_threads(h, threads)
    x = np.zeros(len(b))
    st, res, info = G.gmres_batch_solve(h, b, x, 30, 1e-10, G.ORTHO_MGS, G.MIXED, 20000,
                                        nsys=len(out))
    assert st == G.OK and info.kernel_launches[G.K_BLOCK] == 2
    for i, (A, bi) in enumerate(out):
        xi = x[sys_ptr[i]:sys_ptr[i + 1]]
        assert O.residual_norm(A, bi, xi) / np.linalg.norm(bi) <= 1e-10
    _, oi = O.gmres(out[0][0], out[0][1], m=30, ortho=O.MGS, prec=O.MIXED)
    assert abs(res[0].iters - oi["iters"]) <= max(3, 0.1 * oi["iters"])
    for bad in (0, 100, 2048):
        with pytest.raises(G.GmresError):
            G.gmres_batch_set_cluster_threads(h, bad)
    G.gmres_batch_destroy(h)

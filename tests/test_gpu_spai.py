"""Learned SpAI preconditioner: kernels against the oracle, training, gain,
and the stagnation fallback (marker: gpu).

Binary32 kernels against the binary64 oracle: features (relative 1e-6), M's
values (1e-5 of max |m|), loss (1e-5), dL/dm (1e-4 of max) and the parameter
gradient (1e-3 of max, sums over thousands of nonzeros in binary32), one Adam
step (binary32 rounding).  Then a short training run on small anisotropic
matrices must lower the probe loss and cut the iteration count of a held-out
system against the unpreconditioned and Jacobi-preconditioned mixed solves,
and a poisoned network must still converge through the fallback.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G
    from paper_2011_01850_gb300 import spai as S


def _case(N=6, seed=3):
    A = I.convdiff3d(N, eps=(0.1, 1.0, 10.0), seed=seed)
    n = len(A[0]) - 1
    rng = np.random.default_rng(seed)
    params = (S.jacobi_params() + 0.3 * rng.standard_normal(O.SPAI_NPARAM)).astype(np.float32)
    Z = rng.choice([-1.0, 1.0], size=(4, n)).astype(np.float32)
    return A, n, params, Z


def test_features_parity(gpulib):
    for A in (I.convdiff3d(6, eps=(0.1, 1.0, 10.0), seed=1), I.powerlaw_random(500, seed=2)):
        s = G.Solver(A)
        nnz = len(A[1])
        f = np.zeros(8 * nnz, dtype=np.float32)
        G.gmres_spai_features(s.h, f)
        s.close()
        fo = O.spai_features(A)  # (nnz, 8)
        fg = f.reshape(8, nnz).T
        assert np.allclose(fg, fo, rtol=2e-6, atol=1e-7)


def test_values_parity_and_jacobi(gpulib):
    A, n, params, Z = _case()
    s = G.Solver(A)
    nnz = len(A[1])
    G.gmres_spai_set(s.h, params)
    mg = np.zeros(nnz)
    G.gmres_spai_values(s.h, mg)
    mo = O.spai_values(A, params.astype(np.float64))
    assert np.abs(mg - mo).max() <= 1e-5 * np.abs(mo).max()
    G.gmres_spai_set(s.h, S.jacobi_params())
    G.gmres_spai_values(s.h, mg)
    s.close()
    rp, ci, va = A
    rows = np.repeat(np.arange(n), np.diff(rp))
    d = rows == ci
    assert np.allclose(mg[d], 1.0 / va[d], rtol=2 ** -22)
    assert np.all(mg[~d] == 0.0)


def test_loss_grad_parity(gpulib):
    A, n, params, Z = _case()
    nnz = len(A[1])
    s = G.Solver(A)
    gp = torch.zeros(O.SPAI_NPARAM, device="cuda")
    gm = torch.zeros(nnz, device="cuda")
    Zd = torch.tensor(Z.ravel(), device="cuda")
    loss = G.gmres_spai_loss_grad(s.h, params, Z.shape[0], Zd, gp, gm)
    s.close()
    lo, gpo, gmo = O.spai_loss_grad(A, params.astype(np.float64), Z.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    gm = gm.cpu().numpy()
    assert np.abs(gm - gmo).max() <= 1e-4 * np.abs(gmo).max()
    gp = gp.cpu().numpy()
    assert np.abs(gp - gpo).max() <= 1e-3 * np.abs(gpo).max()
    # layer by layer, relative to the layer's own scale
    for a, b_ in ((0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 4800)):
        assert np.abs(gp[a:b_] - gpo[a:b_]).max() <= 2e-3 * max(np.abs(gpo[a:b_]).max(), 1e-12)


def test_adam_parity(gpulib):
    rng = np.random.default_rng(5)
    p = rng.standard_normal(O.SPAI_NPARAM).astype(np.float32)
    m = (0.1 * rng.standard_normal(O.SPAI_NPARAM)).astype(np.float32)
    v = (0.01 * rng.random(O.SPAI_NPARAM)).astype(np.float32)
    g = rng.standard_normal(O.SPAI_NPARAM).astype(np.float32)
    A = I.convdiff2d(4)
    s = G.Solver(A)
    dp, dm, dv, dg = (torch.tensor(a, device="cuda") for a in (p, m, v, g))
    G.gmres_spai_adam(s.h, dp, dm, dv, dg, 7, 1e-3)
    s.close()
    po, mo, vo = O.adam_step(p, m, v, g, 7, 1e-3)
    # binary32 rounding of each term (the constants 0.9, 0.1, ... included):
    # a few units of 2^-24 of the magnitudes that enter each update
    u = 2.0 ** -24
    m64, g64, v64 = m.astype(np.float64), g.astype(np.float64), v.astype(np.float64)
    assert np.all(np.abs(dm.cpu().numpy() - mo) <= 8 * u * (0.9 * np.abs(m64) + 0.1 * np.abs(g64)))
    assert np.all(np.abs(dv.cpu().numpy() - vo) <= 8 * u * (0.999 * v64 + 0.001 * g64 * g64))
    # (the factors 1 - beta come from binary64, so both moments are tight)
    step = np.abs(po - p.astype(np.float64))
    assert np.all(np.abs(dp.cpu().numpy() - po) <= 8 * u * np.abs(p.astype(np.float64)) + 1e-4 * step)


def test_preconditioned_solve_parity(gpulib):
    """GPU right-preconditioned solve vs the oracle with the same M."""
    A, n, params, Z = _case(N=10)
    p = (S.jacobi_params() + 0.02 * np.random.default_rng(1).standard_normal(
        O.SPAI_NPARAM)).astype(np.float32)
    b = I.rhs_ones_noise(A, 1e-3, 2)
    s = G.Solver(A)
    G.gmres_spai_set(s.h, p)
    mvals = O.spai_values(A, p.astype(np.float64))  # the oracle's own M
    s.set_opts(precond=1, path=G.PATH_GRID)
    x, st, info = s.solve(b, np.zeros(n), m=30, prec="mixed")
    s.close()
    assert st == G.OK and not info["fell_back"]
    rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
    assert rel <= 1e-10
    xo, oi = O.gmres(A, b, m=30, tol=1e-10, ortho=O.CGSR, prec=O.MIXED, maxiter=5000,
                     M=(A[0], A[1], mvals))
    assert abs(info["iters"] - oi["iters"]) <= max(2, oi["iters"] // 10)


@pytest.fixture(scope="module")
def trained():
    A0, _ = S.training_matrix(8, 0)
    tr = S.Trainer(A0)
    for i in range(150):
        A, b = S.training_matrix(8, i)
        tr.train_on(A, b, steps=1, nprobe=8, lr=3e-3, seed=1, use_solver=(i % 10 == 0))
    p = tr.params_host()
    hist = tr.history
    tr.close()
    return p, hist


def _iters(A, b, params=None):
    s = G.Solver(A)
    if params is not None:
        G.gmres_spai_set(s.h, params)
        s.set_opts(precond=1)
    s.set_opts(path=G.PATH_GRID, fallback=0)
    n = len(A[0]) - 1
    x, st, info = s.solve(b, np.zeros(n), m=50, prec="mixed", ortho="cgsr", maxiter=20000)
    s.close()
    assert st == G.OK
    assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
    return info["iters"]


def test_training_lowers_loss(trained):
    p, hist = trained
    assert np.mean(hist[-20:]) < 0.7 * np.mean(hist[:5])


def test_learned_beats_unpreconditioned_and_jacobi(trained):
    """The gain of the trained network on a held-out anisotropic system."""
    p, _ = trained
    A = I.convdiff3d(14, eps=(0.1, 1.0, 10.0), seed=99)
    b = I.rhs_ones_noise(A, 1e-3, 5)
    it_none = _iters(A, b)
    it_jac = _iters(A, b, S.jacobi_params())
    it_learned = _iters(A, b, p)
    assert it_learned < 0.8 * it_none, (it_learned, it_none)
    assert it_learned < 0.8 * it_jac, (it_learned, it_jac)


def test_poisoned_network_falls_back(gpulib):
    A = I.convdiff3d(10, eps=(0.1, 1.0, 10.0), seed=4)
    b = I.rhs_ones_noise(A, 1e-3, 6)
    n = len(A[0]) - 1
    # M = 0 makes no progress at all: the solve must fall back; a network
    # with huge random weights must still end converged (with or without it)
    for poison, must_fall in ((np.zeros(O.SPAI_NPARAM, np.float32), True),
                              ((50 * np.random.default_rng(0).standard_normal(
                                  O.SPAI_NPARAM)).astype(np.float32), False)):
        s = G.Solver(A)
        G.gmres_spai_set(s.h, poison)
        s.set_opts(precond=1, path=G.PATH_GRID)
        x, st, info = s.solve(b, np.zeros(n), m=30, prec="mixed", maxiter=20000)
        s.close()
        assert st == G.OK, info
        assert info["fell_back"] or not must_fall, info
        assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10

"""ILU(0) left preconditioning on the GPU against the oracle (marker: gpu).

The paper's experiments precondition GMRES on the left with ILU(0) (Sec. 4;
Alg. 1: r = M^-1 z, w = M^-1 A v_j).  The factorization and the triangular
solves restate the same eliminations and substitutions in the same order
with separately rounded operations, so in binary64 the factors and M^-1 z
equal the oracle's bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G


def dev(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype or torch.float64)


CASES = [
    ("convdiff2d_33x31", lambda: I.convdiff2d(33, 31, pe=10.0)),
    ("convdiff3d_14", lambda: I.convdiff3d(14, eps=(0.1, 0.1, 0.1), seed=4)),
    ("random_dd_300", lambda: I.random_dd(300, density=0.03, seed=6)),
    ("powerlaw_3000", lambda: I.powerlaw_random(3000, seed=8)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_ilu_factors_bitwise(case, gpulib):
    A = case[1]()
    s = G.Solver(A)
    G.gmres_ilu0(s.h)
    lu = G.gmres_ilu_factors(s.h, len(A[1]))
    s.close()
    assert np.array_equal(lu, O.ilu0(A)[2])


TRSV = [(1, "flags"), (2, "levels"), (3, "wave")]


@pytest.mark.parametrize("trsv", TRSV, ids=[t[1] for t in TRSV])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_ilu_apply(case, trsv, gpulib):
    """Both triangular-solve kernels (per-row ready flags; grid barrier
    between levels) give the oracle's M^-1 z bit for bit in binary64."""
    A = case[1]()
    n = len(A[0]) - 1
    LU = O.ilu0(A)
    z = np.random.default_rng(3).standard_normal(n)
    want = O.ilu_apply(LU, z)
    s = G.Solver(A)
    G.gmres_ilu0(s.h)
    s.set_opts(trsv_kernel=trsv[0])
    out = torch.zeros(n, device="cuda", dtype=torch.float64)
    G.gmres_ilu_apply(s.h, dev(z), out, G.FP64)
    out32 = torch.zeros(n, device="cuda", dtype=torch.float32)
    G.gmres_ilu_apply(s.h, dev(z, torch.float32), out32, G.MIXED)
    s.close()
    scale = np.abs(want).max()
    # binary64: the same subtractions in the same order, separately rounded
    assert np.array_equal(out.cpu().numpy(), want)
    assert np.abs(out32.cpu().numpy() - want).max() <= 1e-4 * scale


@pytest.mark.parametrize("prec", [O.FP64, O.MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("ortho", [O.MGS, O.CGSR], ids=["mgs", "cgsr"])
def test_ilu_cycle_parity(prec, ortho, gpulib):
    A = I.convdiff2d(33, 31, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 4)
    n = len(b)
    s = G.Solver(A)
    G.gmres_ilu0(s.h)
    s.set_opts(precond=G.PRECOND_ILU0)
    g = G.gmres_arnoldi(s.h, dev(b), 24, 12, ortho, {O.FP64: G.FP64, O.MIXED: G.MIXED}[prec], n=n)
    s.close()
    o = O.arnoldi_cycle(A, b, 24, ortho=ortho, prec=prec, kmax=12, ilu=O.ilu0(A))
    tol = {O.FP64: 1e-11, O.MIXED: 2e-4}[prec]
    j = 12
    assert g["j"] == o["j"] == j
    assert np.abs(g["Hbar"][: j + 1, :j] - o["Hbar"][: j + 1, :j]).max() / np.abs(
        o["Hbar"]).max() <= tol
    assert np.abs(g["u"] - o["u"]).max() / np.abs(o["u"]).max() <= tol


@pytest.mark.parametrize("trsv", TRSV, ids=[t[1] for t in TRSV])
@pytest.mark.parametrize("prec", ["fp64", "fp64_ilu32", "mixed", "mixed_limited"])
def test_ilu_solve(prec, trsv, gpulib):
    A = I.convdiff3d(20, eps=(0.1, 0.1, 0.1), seed=2)
    b = I.rhs_ones_noise(A, 1e-3, 6)
    n = len(b)
    s = G.Solver(A)
    _, _, plain = s.solve(b, np.zeros(n), m=40, ortho="cgsr", prec="mixed")
    G.gmres_ilu0(s.h)
    s.set_opts(precond=G.PRECOND_ILU0, ilu_binary32=int(prec == "fp64_ilu32"),
               trsv_kernel=trsv[0])
    p = "fp64" if prec.startswith("fp64") else prec
    x, st, info = s.solve(b, np.zeros(n), m=40, ortho="cgsr", prec=p)
    s.close()
    assert st == G.OK and info["path"] == G.PATH_GRID
    assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
    xl = np.linalg.solve(I.csr_to_dense(A), b)
    assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= 1e-8
    op = {"fp64": O.FP64, "mixed": O.MIXED, "mixed_limited": O.MIXED_LIMITED}[p]
    xo, oi = O.gmres(A, b, m=40, ortho=O.CGSR, prec=op, ilu=O.ilu0(A),
                     ilu32=(prec == "fp64_ilu32"))
    assert abs(info["iters"] - oi["iters"]) <= max(2, 0.1 * oi["iters"]), (info, oi)
    assert info["iters"] < plain["iters"]


def test_ilu_level_counts(gpulib):
    """An N^3 7-point grid in natural order has 3N - 2 dependency levels in
    each triangle (level of (x, y, z) = x + y + z); a 2-D N x M grid has
    N + M - 1; a diagonal matrix has one."""
    for A, want in ((I.convdiff3d(11, eps=(0.1, 0.1, 0.1), seed=1), 31),
                    (I.convdiff2d(9, 13, pe=10.0), 21)):
        s = G.Solver(A)
        with pytest.raises(G.GmresError):
            G.gmres_ilu_levels(s.h)
        G.gmres_ilu0(s.h)
        assert G.gmres_ilu_levels(s.h) == (want, want)
        s.close()
    n = 50
    D = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
         np.linspace(1.0, 2.0, n))
    s = G.Solver(D)
    G.gmres_ilu0(s.h)
    assert G.gmres_ilu_levels(s.h) == (1, 1)
    s.close()


def test_ilu_levels_large_and_short_waits(gpulib):
    """Both triangular-solve kernels on a 3-D stencil wide enough that a
    level spans many warps (48^3: 142 levels of up to 1 700 rows); with a
    one-poll wait limit each either finishes or reports a timeout, and the
    handle keeps working afterwards."""
    A = I.convdiff3d(48, eps=(0.1, 0.1, 0.1), seed=5)
    n = len(A[0]) - 1
    z = np.random.default_rng(9).standard_normal(n)
    want = O.ilu_apply(O.ilu0(A), z)
    s = G.Solver(A)
    G.gmres_ilu0(s.h)
    out = torch.zeros(n, device="cuda", dtype=torch.float64)
    for k in (1, 2, 3, 0):
        s.set_opts(trsv_kernel=k)
        out.zero_()
        G.gmres_ilu_apply(s.h, dev(z), out, G.FP64)
        assert np.array_equal(out.cpu().numpy(), want), k
    for k in (1, 2, 3):
        s.set_opts(trsv_kernel=k, spin_limit=1)
        try:
            G.gmres_ilu_apply(s.h, dev(z), out, G.FP64)
        except G.GmresError as e:
            assert e.status == G.ERR_TIMEOUT
        s.set_opts(spin_limit=0)
        out.zero_()
        G.gmres_ilu_apply(s.h, dev(z), out, G.FP64)
        assert np.array_equal(out.cpu().numpy(), want), k
    s.close()


def test_ilu_refusals_and_timeout(gpulib):
    A = I.convdiff2d(20, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 1)
    n = len(b)
    s = G.Solver(A)
    s.set_opts(precond=G.PRECOND_ILU0)
    with pytest.raises(G.GmresError) as e:  # not factored yet
        s.solve(b, np.zeros(n), m=20, prec="mixed")
    assert e.value.status == G.ERR_ARG
    G.gmres_ilu0(s.h)
    # a spin limit of one poll: the flag-driven triangular solves give up at
    # once and report a timeout; the handle stays usable
    s.set_opts(spin_limit=1, trsv_kernel=1)
    out = torch.zeros(n, device="cuda", dtype=torch.float64)
    with pytest.raises(G.GmresError) as e:
        G.gmres_ilu_apply(s.h, dev(b), out, G.FP64)
    assert e.value.status == G.ERR_TIMEOUT
    s.set_opts(spin_limit=0, trsv_kernel=0)
    x, st, info = s.solve(b, np.zeros(n), m=20, prec="mixed")
    assert st == G.OK
    s.close()
    sp = G.Solver(A, flags=G.CREATE_SPLIT)
    with pytest.raises(G.GmresError):
        G.gmres_ilu0(sp.h)
    sp.close()
    D = I.csr_to_dense(A)
    D[0, 0] = 0.0
    Z = I.dense_to_csr(D)
    sz = G.Solver(Z)
    with pytest.raises(G.GmresError):  # zero pivot
        G.gmres_ilu0(sz.h)
    sz.close()

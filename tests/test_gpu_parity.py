"""CUDA path against the CPU oracle, element by element (marker: gpu).

Kernel level: SpMV (binary64 / binary32, every lanes-per-row variant) and the
binary64 residual, on matrices with empty rows, a 200-entry row, n in
{1, 31, 32, 33, 1000, 4097}.  Cycle level: one restart cycle (basis,
Hessenberg matrix, rotations, s, y, correction) for every precision and both
orthogonalisation schemes.  Solver level: every mode on both paths reaches a
binary64 relative residual <= 1e-10 and matches the oracle's solution.

Tolerances come from the arithmetic: a sum of k products carries at most
gamma_k = k u / (1 - k u) relative error against sum |a||x| for any order of
summation, so two implementations of the same sum differ by at most twice
that; later Arnoldi quantities inherit the per-step error amplified by the
conditioning of the Krylov basis, so the cycle comparisons use a per-precision
tolerance scaled by the step count.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def edge_matrices():
    rng = np.random.default_rng(3)
    out = []
    for n in (1, 31, 32, 33, 1000, 4097):
        out.append(("powerlaw%d" % n, I.powerlaw_random(max(n, 2), seed=n)
                    if n > 1 else I.dense_to_csr(np.array([[2.5]]))))
    # empty rows and one 200-entry row
    n = 700
    D = np.zeros((n, n))
    D[5, rng.choice(n, 200, replace=False)] = rng.standard_normal(200)
    for i in range(n):
        if i % 7 != 3:
            D[i, i] = 3.0
            D[i, (i + 1) % n] = -1.0
    rows = [[] for _ in range(n)]
    rp = [0]
    ci = []
    va = []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        ci += list(nz)
        va += list(D[i, nz])
        rp.append(len(ci))
    out.append(("emptyrows", (np.array(rp, np.int32), np.array(ci, np.int32), np.array(va))))
    out.append(("convdiff3d_12", I.convdiff3d(12, seed=1)))
    return out


@pytest.fixture(scope="module")
def stream():
    torch.cuda.set_device(0)
    return torch.cuda.current_stream()


@pytest.mark.parametrize("name,A", edge_matrices(), ids=[m[0] for m in edge_matrices()])
@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_spmv_parity(name, A, lanes, gpulib, stream):
    rp, ci, va = A
    n = len(rp) - 1
    x = np.random.default_rng(n).standard_normal(n)
    k = np.diff(rp).astype(np.float64)
    absA = (np.abs(va), ci, rp)
    ax = np.zeros(n)
    r = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(ax, r, np.abs(va) * np.abs(x[ci]))
    s = G.Solver(A, stream=stream)
    s.set_opts(spmv_lanes=lanes)
    # binary64
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    G.gmres_spmv(s.h, dev(x), y, G.FP64)
    yo = O.spmv(A, x, O.FP64)
    g = k * U64 / (1 - k * U64)
    assert np.all(np.abs(y.cpu().numpy() - yo) <= 2 * g * ax + 1e-300), name
    # binary32 (values, x and the sum in binary32)
    y32 = torch.zeros(n, dtype=torch.float32, device="cuda")
    G.gmres_spmv(s.h, dev(x, torch.float32), y32, G.MIXED)
    yo32 = O.spmv(A, x, O.MIXED)
    x32 = x.astype(np.float32).astype(np.float64)
    ax32 = np.zeros(n)
    np.add.at(ax32, r, np.abs(va.astype(np.float32)) * np.abs(x32[ci]))
    g32 = k * U32 / (1 - k * U32)
    assert np.all(np.abs(y32.cpu().numpy() - yo32) <= 2 * g32 * ax32 * 1.0001 + 1e-37), name
    s.close()


@pytest.mark.parametrize("name,A", edge_matrices(), ids=[m[0] for m in edge_matrices()])
def test_residual_parity(name, A, gpulib, stream):
    rp, ci, va = A
    n = len(rp) - 1
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n)
    b = rng.standard_normal(n)
    s = G.Solver(A, stream=stream)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    nrm = G.gmres_residual(s.h, dev(b), dev(x), z)
    zo, no = O.residual(A, b, x)
    r = np.repeat(np.arange(n), np.diff(rp))
    ax = np.zeros(n)
    np.add.at(ax, r, np.abs(va) * np.abs(x[ci]))
    k = np.diff(rp) + 1.0
    assert np.all(np.abs(z.cpu().numpy() - zo) <= 2 * k * U64 * (ax + np.abs(b)) * 1.01)
    assert abs(nrm - no) <= 1e-13 * no
    s.close()


# oracle precision codes -> library codes (they differ from MIXED_LIMITED on)
O2G = {O.FP64: 0, O.MIXED: 1, O.MIXED_BF16: 2, O.MIXED_FP16: 3, O.MIXED_LIMITED: 4}

CYCLE_TOL = {O.FP64: 1e-11, O.MIXED: 2e-4, O.MIXED_BF16: 5e-2, O.MIXED_FP16: 2e-2,
             O.MIXED_LIMITED: 1e-4}


@pytest.mark.parametrize("prec", [O.FP64, O.MIXED, O.MIXED_BF16, O.MIXED_FP16, O.MIXED_LIMITED],
                         ids=["fp64", "mixed", "bf16", "fp16", "limited"])
@pytest.mark.parametrize("ortho", [O.MGS, O.CGSR], ids=["mgs", "cgsr"])
def test_cycle_parity(prec, ortho, gpulib, stream):
    """One restart cycle: every exported quantity against the oracle's."""
    A = I.convdiff2d(33, 31, pe=10.0)  # n = 1023: several blocks and a ragged tail
    b = I.rhs_ones_noise(A, 1e-3, 4)
    n = len(A[0]) - 1
    m, kmax = 24, 12
    s = G.Solver(A, stream=stream)
    g = G.gmres_arnoldi(s.h, dev(b), m, kmax, ortho, O2G[prec], n=n)
    o = O.arnoldi_cycle(A, b, m, ortho=ortho, prec=prec, kmax=kmax)
    s.close()
    assert g["j"] == o["j"] == kmax
    tol = CYCLE_TOL[prec]
    j = kmax
    beta = np.linalg.norm(b)

    def close(a, b_, scale, what):
        err = np.abs(a - b_).max() / scale
        assert err <= tol, (what, err, tol)

    close(g["Hbar"][: j + 1, :j], o["Hbar"][: j + 1, :j], np.abs(o["Hbar"]).max(), "Hbar")
    close(g["H"][: j + 1, :j], o["H"][: j + 1, :j], np.abs(o["H"]).max(), "H")
    close(g["cs"][:j], o["cs"][:j], 1.0, "cs")
    close(g["sn"][:j], o["sn"][:j], 1.0, "sn")
    close(g["s"][: j + 1], o["s"][: j + 1], beta, "s")
    close(g["arn"][:j], o["arn"][:j], beta, "arn")
    # v_{j+1} is not formed on the GPU when the cycle ends (the correction
    # uses V_j only), so the basis is compared on its first j vectors
    close(g["V"][:j], o["V"][:j], 1.0 / np.sqrt(n) * 10, "V")
    close(g["u"], o["u"], np.abs(o["u"]).max(), "u")
    # the first basis vector is r0/beta rounded to the basis: equal up to one
    # rounding of the quotient (the two betas differ in the last place)
    v1o = O.round_basis(b / beta, prec, n)
    assert np.allclose(g["V"][0], v1o, rtol=(4e-3 if prec >= O.MIXED_BF16 else 1e-6),
                       atol=1e-300)


def _solve(A, b, prec, ortho, path, m=30, tol=1e-10, stream=None, maxiter=4000):
    s = G.Solver(A, stream=stream)
    s.set_opts(path=path)
    n = len(A[0]) - 1
    db = dev(b)
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    x, st, info = s.solve(db, dx, m=m, tol=tol, ortho=ortho, prec=prec, maxiter=maxiter)
    s.close()
    return dx.cpu().numpy(), st, info


SOLVE_CASES = [
    ("convdiff2d_40", lambda: I.convdiff2d(40, pe=10.0)),
    ("powerlaw_3000", lambda: I.powerlaw_random(3000, seed=12)),
    ("convdiff3d_14", lambda: I.convdiff3d(14, seed=2)),
]


@pytest.mark.parametrize("case", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16", "mixed_fp16"])
@pytest.mark.parametrize("ortho", ["mgs", "cgsr"])
@pytest.mark.parametrize("path", [1, 2], ids=["grid", "block"])
def test_solve_parity(case, prec, ortho, path, gpulib, stream):
    A = case[1]()
    b = I.rhs_ones_noise(A, 1e-3, 11)
    x, st, info = _solve(A, b, prec, ortho, path, stream=stream)
    assert st == G.OK, info
    rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
    assert rel <= 1e-10, (rel, info)
    assert abs(rel - info["relres"]) <= 1e-3 * rel + 1e-14
    xo, _ = O.gmres(A, b, m=30, tol=1e-13, ortho=O.CGSR, prec=O.FP64, maxiter=20000)
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    # forward error of any x with relative residual rel is at most kappa*rel,
    # so 1e-8 is the bar wherever kappa * 1e-10 <= 1e-8, else kappa bounds it
    kappa = _kappa(case[0], A)
    assert err <= max(1e-8, 2 * kappa * (rel + 1e-13)), (err, kappa, rel)
    if kappa * 1e-10 <= 1e-8:
        assert err <= 1e-8, err


@pytest.mark.parametrize("case", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
@pytest.mark.parametrize("ortho", ["mgs", "cgsr"])
def test_limited_solve_parity(case, ortho, gpulib, stream):
    """Limited mixed precision (Sec. 4.1; grid path): the binary64 target and
    the oracle's solution, as for the other modes; the block path refuses it."""
    A = case[1]()
    b = I.rhs_ones_noise(A, 1e-3, 11)
    x, st, info = _solve(A, b, "mixed_limited", ortho, 1, stream=stream)
    assert st == G.OK, info
    rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
    assert rel <= 1e-10, (rel, info)
    xo, oi = O.gmres(A, b, m=30, tol=1e-13, ortho=O.CGSR, prec=O.FP64, maxiter=20000)
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    kappa = _kappa(case[0], A)
    assert err <= max(1e-8, 2 * kappa * (rel + 1e-13)), (err, kappa, rel)
    with pytest.raises(G.GmresError) as e:
        _solve(A, b, "mixed_limited", ortho, 2, stream=stream)
    assert e.value.status == G.ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("ortho", ["mgs", "cgsr"])
def test_block_cluster_single_system(prec, ortho, gpulib, stream):
    """The block path on one cluster of 8 blocks (reductions through
    distributed shared memory) against one block: both reach the binary64
    target, agree with the oracle, and binary64 takes the same schedule."""
    A = I.convdiff2d(64, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 7)
    n = len(b)
    out = {}
    for cs in (1, 8):
        s = G.Solver(A, stream=stream)
        s.set_opts(path=G.PATH_BLOCK, block_cluster=cs)
        x, st, info = s.solve(b, np.zeros(n), m=50, ortho=ortho, prec=prec)
        s.close()
        assert st == G.OK
        assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
        out[cs] = (x, info)
    xo, oi = O.gmres(A, b, m=50, tol=1e-10, ortho=O.MGS if ortho == "mgs" else O.CGSR,
                     prec=O.FP64 if prec == "fp64" else O.MIXED)
    if prec == "fp64":
        assert out[8][1]["iters"] == out[1][1]["iters"] == oi["iters"]
        assert np.linalg.norm(out[8][0] - xo) / np.linalg.norm(xo) <= 1e-11


def test_limited_takes_fewer_iterations_than_mixed(gpulib, stream):
    """Sec. 4.1: limiting binary32 to A, M and the basis lets MGS improve
    further before it stalls, so the limited solver needs no more inner
    iterations than the fully mixed one (and its cycles use binary64
    vectors: the workspace is the binary64 one with a binary32 basis)."""
    A = I.convdiff2d(30, pe=1.0)
    b = I.rhs_ones_noise(A, 1e-3, 1)
    s = G.Solver(A, stream=stream)
    s.set_opts(path=G.PATH_GRID)
    _, st1, i1 = s.solve(b, np.zeros(len(b)), m=100, ortho="mgs", prec="mixed")
    _, st2, i2 = s.solve(b, np.zeros(len(b)), m=100, ortho="mgs", prec="mixed_limited")
    _, w64 = G.gmres_memory_bytes(s.h, 100, G.FP64)
    _, wlim = G.gmres_memory_bytes(s.h, 100, G.MIXED_LIMITED)
    s.close()
    assert st1 == st2 == G.OK
    assert i2["iters"] <= i1["iters"], (i1["iters"], i2["iters"])
    xo, oi = O.gmres(A, b, m=100, ortho=O.MGS, prec=O.MIXED_LIMITED)
    assert abs(i2["iters"] - oi["iters"]) <= 0.25 * oi["iters"]
    ldv = ((len(b) + 2047) // 2048) * 2048
    assert w64 - wlim == 101 * ldv * 4


def test_precision_changes_on_one_handle(gpulib, stream):
    """Solves of different working precisions in a row on one handle (grid
    path, n not a multiple of the padding): the padding rows of the work
    vectors are cleared when the working type changes, so every solve still
    reaches the binary64 target."""
    A = I.convdiff2d(40, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 5)
    n = len(b)
    s = G.Solver(A, stream=stream)
    s.set_opts(path=G.PATH_GRID)
    for prec in ("fp64", "mixed", "mixed_limited", "mixed_bf16", "fp64", "mixed_fp16"):
        x, st, info = s.solve(b, np.zeros(n), m=30, ortho="cgsr", prec=prec)
        assert st == G.OK, prec
        assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10, prec
    s.close()


def test_backward_error(gpulib, stream):
    """The normwise backward error the paper reports (infinity-norm form)
    against numpy's, on the solution of a mixed solve and on x = 0 (where it
    is ||b|| / ||b|| = 1), also with split storage."""
    A = I.convdiff2d(40, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 5)
    n = len(b)
    D = I.csr_to_dense(A)
    for flags in (0, G.CREATE_SPLIT):
        s = G.Solver(A, flags=flags, stream=stream)
        db = dev(b)
        dx = torch.zeros(n, dtype=torch.float64, device="cuda")
        assert G.gmres_backward_error(s.h, db, dx) == 1.0
        s.solve(db, dx, m=30, ortho="cgsr", prec="mixed")
        eta = G.gmres_backward_error(s.h, db, dx)
        s.close()
        x = dx.cpu().numpy()
        want = np.abs(b - D @ x).max() / (np.abs(D).sum(axis=1).max() * np.abs(x).max()
                                          + np.abs(b).max())
        assert 0 < eta <= 1e-10 and abs(eta - want) <= 1e-3 * want, (eta, want)


_KAPPA = {}


def _kappa(name, A):
    if name not in _KAPPA:
        _KAPPA[name] = np.linalg.cond(I.csr_to_dense(A))
    return _KAPPA[name]


def test_solve_matches_oracle_iterations_fp64(gpulib, stream):
    """Binary64: the GPU and the oracle take the same restart schedule."""
    A = I.convdiff2d(24, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 2)
    for path in (1, 2):
        for ortho, oo in (("mgs", O.MGS), ("cgsr", O.CGSR)):
            x, st, info = _solve(A, b, "fp64", ortho, path, m=20, stream=stream)
            xo, oi = O.gmres(A, b, m=20, tol=1e-10, ortho=oo, prec=O.FP64, maxiter=4000)
            assert info["restarts"] == oi["restarts"] and info["iters"] == oi["iters"]
            assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-11


def test_host_buffers_equal_device_buffers(gpulib, stream):
    A = I.convdiff2d(30, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 3)
    n = len(A[0]) - 1
    s = G.Solver(A, stream=stream)
    s.set_opts(path=G.PATH_GRID)
    xh = np.zeros(n)
    _, st1, i1 = s.solve(b, xh, m=25, prec="mixed")
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, st2, i2 = s.solve(dev(b), dx, m=25, prec="mixed")
    s.close()
    assert st1 == st2 == G.OK
    assert np.array_equal(xh, dx.cpu().numpy())  # deterministic reductions


def test_repeatable_bitwise(gpulib, stream):
    A = I.powerlaw_random(5000, seed=9)
    b = I.rhs_ones_noise(A, 1e-3, 1)
    x1, _, _ = _solve(A, b, "mixed", "cgsr", 1, stream=stream)
    x2, _, _ = _solve(A, b, "mixed", "cgsr", 1, stream=stream)
    assert np.array_equal(x1, x2)


def test_edge_cases(gpulib, stream):
    A = I.convdiff2d(10, pe=10.0)
    n = len(A[0]) - 1
    s = G.Solver(A, stream=stream)
    # b = 0 -> x = 0, converged
    for path in (1, 2):
        s.set_opts(path=path)
        x = np.ones(n)
        _, st, info = s.solve(np.zeros(n), x)
        assert st == G.OK and np.all(x == 0)
    # maxiter = 0 -> iteration limit (x untouched)
    s.set_opts(path=1)
    x = np.zeros(n)
    _, st, info = s.solve(np.ones(n), x, maxiter=0)
    assert st == G.MAXITER and info["iters"] == 0
    # NaN in b
    bad = np.ones(n)
    bad[3] = np.nan
    with pytest.raises(G.GmresError) as e:
        s.solve(bad, np.zeros(n))
    assert e.value.status == G.ERR_NONFINITE
    # bad arguments
    for kw in (dict(m=0), dict(m=129), dict(tol=0.0), dict(maxiter=-1)):
        with pytest.raises(G.GmresError) as e:
            s.solve(np.ones(n), np.zeros(n), **kw)
        assert e.value.status == G.ERR_ARG
    s.close()
    # invalid CSR / non-finite values are rejected at create time
    rp, ci, va = A
    ci2 = ci.copy()
    ci2[0] = n
    with pytest.raises(G.GmresError) as e:
        G.Solver((rp, ci2, va))
    assert e.value.status == G.ERR_ARG
    va2 = va.copy()
    va2[1] = np.inf
    with pytest.raises(G.GmresError) as e:
        G.Solver((rp, ci, va2))
    assert e.value.status == G.ERR_NONFINITE
    # 1 x 1 system
    one = I.dense_to_csr(np.array([[4.0]]))
    for path in (1, 2):
        x, st, info = _solve(one, np.array([2.0]), "mixed", "mgs", path, stream=stream)
        assert st == G.OK and abs(x[0] - 0.5) < 1e-12


def test_memory_model(gpulib, stream):
    """Device footprint follows the paper's storage model (Sec. 4) without the
    ILU factors: the matrix keeps shared int32 indices plus binary64 and
    binary32 values; the basis costs (m+1) n s_V bytes."""
    A = I.convdiff2d(50, pe=10.0)
    n, nnz = len(A[0]) - 1, len(A[1])
    s = G.Solver(A, stream=stream)
    mb, wb64 = G.gmres_memory_bytes(s.h, 50, G.FP64)
    _, wb32 = G.gmres_memory_bytes(s.h, 50, G.MIXED)
    _, wb16 = G.gmres_memory_bytes(s.h, 50, G.MIXED_BF16)
    s.close()
    assert mb == 16 * nnz + 4 * (n + 1)
    ldv = ((n + 2047) // 2048) * 2048
    assert wb64 - wb32 >= 51 * ldv * 4
    assert wb32 - wb16 == 51 * ldv * 2


def test_mgs_cooperative_matches_per_column(gpulib, stream):
    """The cooperative MGS kernel (w in shared memory, one launch per step)
    and the per-basis-vector kernels agree: binary64 takes the same schedule
    and solutions agree to 1e-11; mixed both reach the binary64 target."""
    A = I.powerlaw_random(60000, seed=21)
    b = I.rhs_ones_noise(A, 1e-3, 3)
    n = len(A[0]) - 1
    out = {}
    for kern in (0, 1):
        for prec in ("fp64", "mixed_bf16"):
            s = G.Solver(A, stream=stream)
            s.set_opts(path=G.PATH_GRID, mgs_kernel=kern)
            x, st, info = s.solve(b, np.zeros(n), m=40, ortho="mgs", prec=prec)
            s.close()
            assert st == G.OK
            assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
            out[(kern, prec)] = (x, info)
    x0, i0 = out[(0, "fp64")]
    x1, i1 = out[(1, "fp64")]
    assert i0["iters"] == i1["iters"] and i0["restarts"] == i1["restarts"]
    assert np.linalg.norm(x0 - x1) / np.linalg.norm(x1) <= 1e-11
    assert i0["kernel_launches"]["ortho"] < i1["kernel_launches"]["ortho"]


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16", "mixed_fp16"])
@pytest.mark.parametrize("n", [60000, 2_000_000])
def test_mgs_staged_equals_unstaged(prec, n, gpulib, stream):
    """The cooperative MGS kernel with the basis rows staged in shared memory
    by bulk copies (mgs_kernel 0) does the unstaged kernel's arithmetic in
    the same order (mgs_kernel 2): one restart cycle gives the same Hessenberg
    matrix, basis and correction bit for bit, at a size where every block
    holds a short row chunk and at the power-law workload's 2 M rows (binary64
    there too large to stage: both run unstaged, still equal)."""
    A = I.powerlaw_random(n, seed=21)
    b = I.rhs_ones_noise(A, 1e-3, 3)
    res = []
    for kern in (0, 2):
        s = G.Solver(A, stream=stream)
        s.set_opts(path=G.PATH_GRID, mgs_kernel=kern)
        res.append(G.gmres_arnoldi(s.h, dev(b), 50, 50, G.ORTHO_MGS, G.PRECISIONS[prec], n=n))
        s.close()
    g0, g2 = res
    assert g0["j"] == g2["j"] == 50
    for k in ("Hbar", "H", "s", "y", "u", "V"):
        assert np.array_equal(g0[k], g2[k]), k


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_fp16"])
def test_cgsr_kernel_families_agree(prec, gpulib, stream):
    """The CGSR kernel families (rows with the update split by basis vectors
    and pass B's slice in registers; rows with the update split by rows) sum
    in different orders; binary64 takes the same schedule with solutions
    equal to 1e-11, and both reach the binary64 target.  The retired
    families are rejected."""
    A = I.convdiff3d(26, eps=(0.1, 0.1, 0.1), seed=3)  # n = 17576: several slices per block
    b = I.rhs_ones_noise(A, 1e-3, 5)
    n = len(A[0]) - 1
    out = {}
    for kern in (0, 2):
        s = G.Solver(A, stream=stream)
        s.set_opts(path=G.PATH_GRID, cgs_kernel=kern)
        x, st, info = s.solve(b, np.zeros(n), m=40, ortho="cgsr", prec=prec)
        s.close()
        assert st == G.OK
        assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
        out[kern] = (x, info)
    s = G.Solver(A, stream=stream)
    for kern in (1, 3):
        with pytest.raises(G.GmresError):
            s.set_opts(cgs_kernel=kern)
    s.close()
    if prec == "fp64":
        for kern in (2,):
            assert out[kern][1]["iters"] == out[0][1]["iters"]
            assert out[kern][1]["restarts"] == out[0][1]["restarts"]
            assert np.linalg.norm(out[kern][0] - out[0][0]) / np.linalg.norm(out[0][0]) <= 1e-11


def test_bounded_wait_reports_timeout(gpulib, stream):
    """With the spin limit at 1 the exchange waits of the cooperative MGS
    kernel give up at once: the solve ends with GMRES_ERR_TIMEOUT instead of
    waiting, and the handle stays usable."""
    A = I.powerlaw_random(200000, seed=5)
    b = I.rhs_ones_noise(A, 1e-3, 4)
    n = len(A[0]) - 1
    s = G.Solver(A, stream=stream)
    s.set_opts(path=G.PATH_GRID, mgs_kernel=0, spin_limit=1)
    with pytest.raises(G.GmresError) as e:
        s.solve(b, np.zeros(n), m=10, ortho="mgs", prec="mixed")
    assert e.value.status == G.ERR_TIMEOUT
    s.set_opts(spin_limit=0)
    x, st, info = s.solve(b, np.zeros(n), m=30, ortho="mgs", prec="mixed")
    s.close()
    assert st == G.OK
    assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10

"""A stored once, split into the high- and low-order 32 bits of each binary64
value (Sec. 4 outlook; marker: gpu).

The binary32 Krylov step reads the high part (the value with its low 32 bits
cleared), binary64 work reads both parts; 8 bytes per nonzero instead of the
12 of a binary64 plus a binary32 copy."""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G


def dev(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), device="cuda",
                        dtype=dtype or torch.float64)


def _high(v):
    u = np.ascontiguousarray(v, dtype=np.float64).view(np.uint64) & np.uint64(0xFFFFFFFF00000000)
    return u.view(np.float64)


def test_split_memory_and_spmv(gpulib):
    A = I.convdiff2d(40, pe=10.0)
    n, nnz = len(A[0]) - 1, len(A[1])
    s = G.Solver(A, flags=G.CREATE_SPLIT)
    ref = G.Solver(A)
    mb, _ = G.gmres_memory_bytes(s.h, 30, G.MIXED)
    mr, _ = G.gmres_memory_bytes(ref.h, 30, G.MIXED)
    assert mb == 4 * (n + 1) + 12 * nnz and mr - mb == 4 * nnz
    x = np.random.default_rng(1).standard_normal(n)
    # binary64 SpMV reads both halves: the exact values, bit for bit as unsplit
    y64, r64 = torch.zeros(n, device="cuda", dtype=torch.float64), torch.zeros(
        n, device="cuda", dtype=torch.float64)
    G.gmres_spmv(s.h, dev(x), y64, G.FP64)
    G.gmres_spmv(ref.h, dev(x), r64, G.FP64)
    assert torch.equal(y64, r64)
    # binary32 SpMV reads the high half: A_hi (numpy bit masking) within
    # the binary32 sum bound
    x32 = x.astype(np.float32)
    y32 = torch.zeros(n, device="cuda", dtype=torch.float32)
    G.gmres_spmv(s.h, dev(x32, torch.float32), y32, G.MIXED)
    Ahi = _high(I.csr_to_dense(A))
    want = Ahi @ x32.astype(np.float64)
    bound = 2 * 8 * 2.0 ** -24 * (np.abs(Ahi) @ np.abs(x32.astype(np.float64))) + 1e-30
    assert np.all(np.abs(y32.cpu().numpy() - want) <= bound)
    s.close()
    ref.close()


@pytest.mark.parametrize("prec", [O.FP64, O.MIXED, O.MIXED_LIMITED],
                         ids=["fp64", "mixed", "limited"])
@pytest.mark.parametrize("ortho", [O.MGS, O.CGSR], ids=["mgs", "cgsr"])
def test_split_cycle_parity(prec, ortho, gpulib):
    """One restart cycle on split storage against the oracle's split cycle."""
    A = I.convdiff2d(33, 31, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 4)
    n = len(b)
    gprec = {O.FP64: G.FP64, O.MIXED: G.MIXED, O.MIXED_LIMITED: G.MIXED_LIMITED}[prec]
    s = G.Solver(A, flags=G.CREATE_SPLIT)
    g = G.gmres_arnoldi(s.h, dev(b), 24, 12, ortho, gprec, n=n)
    s.close()
    o = O.arnoldi_cycle(A, b, 24, ortho=ortho, prec=prec, kmax=12, split_bytes=True)
    tol = {O.FP64: 1e-11, O.MIXED: 2e-4, O.MIXED_LIMITED: 1e-4}[prec]
    j = 12
    assert g["j"] == o["j"] == j
    scale = np.abs(o["Hbar"]).max()
    assert np.abs(g["Hbar"][: j + 1, :j] - o["Hbar"][: j + 1, :j]).max() / scale <= tol
    assert np.abs(g["u"] - o["u"]).max() / np.abs(o["u"]).max() <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16", "mixed_limited"])
def test_split_solve(prec, gpulib):
    """Every precision reaches the binary64 target on split storage; binary64
    is bitwise the unsplit solve."""
    A = I.convdiff3d(20, eps=(0.1, 0.1, 0.1), seed=2)
    b = I.rhs_ones_noise(A, 1e-3, 6)
    n = len(b)
    s = G.Solver(A, flags=G.CREATE_SPLIT)
    x, st, info = s.solve(b, np.zeros(n), m=40, ortho="cgsr", prec=prec)
    s.close()
    assert st == G.OK and info["path"] == G.PATH_GRID
    assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
    xo, oi = O.gmres(A, b, m=40, tol=1e-10, ortho=O.CGSR,
                     prec={"fp64": O.FP64, "mixed": O.MIXED, "mixed_bf16": O.MIXED_BF16,
                           "mixed_limited": O.MIXED_LIMITED}[prec], split_bytes=True)
    assert abs(info["iters"] - oi["iters"]) <= max(2, 0.1 * oi["iters"])
    if prec == "fp64":
        r = G.Solver(A)
        r.set_opts(path=G.PATH_GRID)
        x2, st2, i2 = r.solve(b, np.zeros(n), m=40, ortho="cgsr", prec=prec)
        r.close()
        assert np.array_equal(x, x2) and i2["iters"] == info["iters"]


def test_split_refusals(gpulib):
    A = I.convdiff2d(20, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 1)
    with pytest.raises(G.GmresError):
        G.Solver(A, flags=G.CREATE_SPLIT | G.CREATE_TRANSPOSE)
    s = G.Solver(A, flags=G.CREATE_SPLIT)
    s.set_opts(path=G.PATH_BLOCK)
    with pytest.raises(G.GmresError) as e:
        s.solve(b, np.zeros(len(b)), m=20, prec="mixed")
    assert e.value.status == G.ERR_ARG
    with pytest.raises(G.GmresError):
        G.gmres_spai_set(s.h, dev(np.zeros(G.SPAI_NPARAM), torch.float32))
    s.close()

"""A in sliced storage (gmres_opts.spmv_format) on the GPU (marker: gpu).

The sliced product (slices of 32 rows stored column-major, sell.cuh) sums
every row in the order and grouping of the CSR kernel at one lane per row, so
it must give the same bits: checked for the plain product (also against the
oracle's rounding bound), for a whole restart cycle of every precision and
orthogonalisation, and for whole solves.  Also: the choice of 16-bit column
offsets or 32-bit columns (through the device bytes the copy holds), the
refill after gmres_set_values, the refusal with split storage, and the
autotuner's report.
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


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def _matrices():
    rng = np.random.default_rng(7)
    out = [("one", I.dense_to_csr(np.array([[2.5]])))]
    for n in (31, 33, 1000):
        out.append(("powerlaw%d" % n, I.powerlaw_random(n, seed=n)))
    # empty rows, one 300-entry row and a ragged last slice
    n = 709
    D = np.zeros((n, n))
    D[5, rng.choice(n, 300, replace=False)] = rng.standard_normal(300)
    for i in range(n):
        if i % 7 != 3:
            D[i, i] = 3.0
            D[i, (i + 1) % n] = -1.0
    out.append(("emptyrows", I.dense_to_csr(D)))
    out.append(("convdiff3d_12", I.convdiff3d(12, seed=1)))
    # columns up to 50 000 rows away: 32-bit column storage
    out.append(("powerlaw50000", I.powerlaw_random(50000, seed=4)))
    return out


MATS = _matrices()


def _sliced_bytes(A, idx_bytes):
    rp = np.asarray(A[0], np.int64)
    n = len(rp) - 1
    nsl = (n + 31) // 32
    lens = np.zeros(nsl * 32, np.int64)
    lens[:n] = np.diff(rp)
    ent = int((32 * lens.reshape(nsl, 32).max(axis=1)).sum())
    return 4 * (nsl + 1) + 2 * nsl * 32 + ent * (idx_bytes + 4 + 8)


def _products(s, x, n):
    y64 = torch.zeros(n, dtype=torch.float64, device="cuda")
    G.gmres_spmv(s.h, _dev(x), y64, G.FP64)
    y32 = torch.zeros(n, dtype=torch.float32, device="cuda")
    G.gmres_spmv(s.h, _dev(x, torch.float32), y32, G.MIXED)
    return y64, y32


@pytest.mark.parametrize("name,A", MATS, ids=[m[0] for m in MATS])
def test_sliced_spmv_equals_csr(name, A, gpulib):
    rp, ci, va = A
    n = len(rp) - 1
    x = np.random.default_rng(n).standard_normal(n)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    s.set_opts(spmv_format=G.SPMV_CSR, spmv_lanes=1)
    base = G.gmres_memory_bytes(s.h, 10, G.FP64)[0]
    c64, c32 = _products(s, x, n)
    s.set_opts(spmv_format=G.SPMV_SLICED)
    assert G.gmres_spmv_format(s.h) == (G.SPMV_SLICED, G.SPMV_SLICED)
    # 16-bit offsets exactly when every |col - row| fits
    r = np.repeat(np.arange(n), np.diff(rp))
    idx = 2 if (len(ci) == 0 or np.abs(ci.astype(np.int64) - r).max() <= 32767) else 4
    assert G.gmres_memory_bytes(s.h, 10, G.FP64)[0] - base == _sliced_bytes(A, idx), name
    y64, y32 = _products(s, x, n)
    s.close()
    assert torch.equal(y64, c64), name
    assert torch.equal(y32, c32), name
    # and within the oracle's rounding bound (binary64: 2 gamma_k |A||x| per row)
    k = np.diff(rp).astype(np.float64)
    ax = np.zeros(n)
    np.add.at(ax, r, np.abs(va) * np.abs(x[ci]))
    g = k * U64 / (1 - k * U64)
    assert np.all(np.abs(y64.cpu().numpy() - O.spmv(A, x, O.FP64)) <= 2 * g * ax + 1e-300)
    x32 = x.astype(np.float32).astype(np.float64)
    ax32 = np.zeros(n)
    np.add.at(ax32, r, np.abs(va.astype(np.float32)) * np.abs(x32[ci]))
    g32 = k * U32 / (1 - k * U32)
    assert np.all(np.abs(y32.cpu().numpy() - O.spmv(A, x, O.MIXED))
                  <= 2 * g32 * ax32 * 1.0001 + 1e-37)


CYCLE_MATS = [("convdiff3d_16", I.convdiff3d(16, seed=3)),
              ("powerlaw5000", I.powerlaw_random(5000, seed=5)),
              ("powerlaw40000", I.powerlaw_random(40000, seed=6))]


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16", "mixed_fp16"])
@pytest.mark.parametrize("ortho", [O.MGS, O.CGSR], ids=["mgs", "cgsr"])
@pytest.mark.parametrize("name,A", CYCLE_MATS, ids=[m[0] for m in CYCLE_MATS])
def test_sliced_cycle_equals_csr(name, A, ortho, prec, gpulib):
    """One restart cycle through the C-ABI: every exported array bit for bit."""
    b = I.rhs_ones_noise(A, 1e-3, 2)
    n = len(b)
    out = {}
    s = G.Solver(A, stream=torch.cuda.current_stream())
    for fmt in (G.SPMV_CSR, G.SPMV_SLICED):
        s.set_opts(spmv_format=fmt, spmv_lanes=1)
        out[fmt] = G.gmres_arnoldi(s.h, _dev(b), 40, 25, ortho, G.PRECISIONS[prec], n=n)
    s.close()
    a, c = out[G.SPMV_CSR], out[G.SPMV_SLICED]
    assert a["j"] == c["j"]
    for key, v in a.items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, c[key], equal_nan=True), (name, prec, key)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_bf16"])
def test_sliced_solve_equals_csr(prec, gpulib):
    A = I.convdiff3d(24, seed=2)
    b = I.rhs_ones_noise(A, 1e-3, 9)
    n = len(b)
    res = {}
    s = G.Solver(A, stream=torch.cuda.current_stream())
    for fmt in (G.SPMV_CSR, G.SPMV_SLICED):
        s.set_opts(spmv_format=fmt, spmv_lanes=1)
        dx = torch.zeros(n, dtype=torch.float64, device="cuda")
        _, st, info = s.solve(_dev(b), dx, m=50, tol=1e-10, ortho="cgsr", prec=prec,
                              maxiter=5000)
        assert st == G.OK
        res[fmt] = (dx.cpu().numpy(), info["iters"], info["relres"])
    s.close()
    (x0, i0, r0), (x1, i1, r1) = res[G.SPMV_CSR], res[G.SPMV_SLICED]
    assert i0 == i1 and r0 == r1
    assert np.array_equal(x0, x1)
    assert O.residual_norm(A, b, x1) / np.linalg.norm(b) <= 1e-10


def test_sliced_refill_after_set_values(gpulib):
    A = I.convdiff3d(10, seed=1)
    rp, ci, va = A
    n = len(rp) - 1
    x = np.random.default_rng(1).standard_normal(n)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    s.set_opts(spmv_format=G.SPMV_SLICED, spmv_lanes=1)
    va2 = va * (1.5 + np.random.default_rng(2).random(len(va)))
    G.gmres_set_values(s.h, va2)
    y64, y32 = _products(s, x, n)
    s.set_opts(spmv_format=G.SPMV_CSR)
    c64, c32 = _products(s, x, n)
    s.close()
    assert torch.equal(y64, c64) and torch.equal(y32, c32)
    assert np.allclose(y64.cpu().numpy(), O.spmv((rp, ci, va2), x, O.FP64), rtol=1e-13,
                       atol=1e-13)


def test_sliced_refused_with_split_storage(gpulib):
    A = I.convdiff3d(8, seed=1)
    s = G.Solver(A, flags=G.CREATE_SPLIT, stream=torch.cuda.current_stream())
    with pytest.raises(G.GmresError) as e:
        s.set_opts(spmv_format=G.SPMV_SLICED)
    assert e.value.status == G.ERR_ARG
    assert G.gmres_spmv_format(s.h) == (G.SPMV_CSR, G.SPMV_CSR)
    with pytest.raises(G.GmresError):
        s.set_opts(spmv_format=3)
    s.close()


def test_autotune_reports_the_storage(gpulib):
    A = I.convdiff3d(48, seed=2)
    b = I.rhs_ones_noise(A, 1e-3, 3)
    n = len(b)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    assert G.gmres_spmv_format(s.h) == (G.SPMV_CSR, G.SPMV_CSR)  # before the autotuner
    G.gmres_autotune(s.h)
    f32, f64 = G.gmres_spmv_format(s.h)
    assert f32 in (G.SPMV_CSR, G.SPMV_SLICED) and f64 in (G.SPMV_CSR, G.SPMV_SLICED)
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, st, _ = s.solve(_dev(b), dx, m=50, tol=1e-10, ortho="cgsr", prec="mixed")
    assert st == G.OK
    s.set_opts(spmv_format=G.SPMV_CSR)
    assert G.gmres_spmv_format(s.h) == (G.SPMV_CSR, G.SPMV_CSR)
    s.set_opts(spmv_format=G.SPMV_AUTO)
    assert G.gmres_spmv_format(s.h) == (f32, f64)
    s.close()
    assert O.residual_norm(A, b, dx.cpu().numpy()) / np.linalg.norm(b) <= 1e-10

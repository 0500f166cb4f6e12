"""The synthetic inputs have the structure their recipes state (CPU).

They stand in for the paper's SuiteSparse matrices: the 2-D and 3-D
first-order upwind convection-diffusion stencils (5 and 7 points, Dirichlet
boundary), the random matrix with power-law row lengths (3..200, exponent
1.734, mean 16, diagonal 1.2 x the off-diagonal absolute row sum), the batch
of uneven 2-D systems (sizes log-uniform in [500, 50000]) and b = A 1 + noise
(sigma 1e-3).  Every generator is seeded: the same seed gives the same
arrays, another seed other ones.
"""
import numpy as np

from paper_2011_01850_gb300 import inputs as I


def rows_of(A):
    rp = A[0]
    return np.repeat(np.arange(len(rp) - 1), np.diff(rp))


def check_csr(A):
    rp, ci, va = A
    n = len(rp) - 1
    assert rp[0] == 0 and np.all(np.diff(rp) >= 1) and rp[-1] == len(ci) == len(va)
    assert ci.min() >= 0 and ci.max() < n
    for i in range(0, n, max(1, n // 257)):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0), i  # sorted, distinct
    r = rows_of(A)
    assert np.array_equal(np.bincount(r[ci == r], minlength=n), np.ones(n))  # one diagonal


def test_stencil_patterns():
    for N in (1, 2, 12):
        A = I.convdiff3d(N, eps=(0.1, 0.1, 0.1), seed=3)
        check_csr(A)
        assert len(A[1]) == 7 * N ** 3 - 6 * N ** 2
    for nx, ny in ((1, 1), (9, 13), (64, 64)):
        A = I.convdiff2d(nx, ny, pe=10.0)
        check_csr(A)
        assert len(A[1]) == 5 * nx * ny - 2 * (nx + ny)
    # first-order upwind with positive diffusion: positive diagonal,
    # non-positive off-diagonals, weak row diagonal dominance
    for A in (I.convdiff3d(10, eps=(0.1, 1.0, 10.0), seed=4), I.convdiff2d(20, pe=50.0)):
        rp, ci, va = A
        r = rows_of(A)
        diag = va[ci == r]
        off = np.bincount(r[ci != r], weights=np.abs(va[ci != r]), minlength=len(rp) - 1)
        assert np.all(diag > 0) and np.all(va[ci != r] <= 0)
        assert np.all(diag >= off * (1 - 1e-12))


def test_full_size_stencil_counts():
    # the 160^3 matrix of the benchmark: n = 4 096 000, nnz = 28 518 400
    assert 7 * 160 ** 3 - 6 * 160 ** 2 == 28_518_400


def test_powerlaw_recipe():
    A = I.powerlaw_random(200_000, seed=11)
    check_csr(A)
    rp, ci, va = A
    L = np.diff(rp)
    assert L.min() == 3 and L.max() == 200
    assert abs(L.mean() - 16.0) < 0.3
    assert abs((L == 3).mean() - 0.225) < 0.005
    assert abs((L >= 100).mean() - 0.028) < 0.003
    r = rows_of(A)
    off = ci != r
    d = va[~off]
    s = np.bincount(r[off], weights=np.abs(va[off]), minlength=len(rp) - 1)
    assert np.allclose(d, 1.2 * s, rtol=1e-14, atol=0)
    assert abs(va[off].mean()) < 0.01 and abs(va[off].var() - 1.0) < 0.01


def test_batch_recipe():
    sy = I.batched_convdiff2d(count=2048, nmin=500, nmax=50000, seed=20110185)
    ns = np.array([len(b) for _, b in sy])
    assert len(sy) == 2048
    assert ns.min() >= 450 and ns.max() <= 50_500  # rounding of the grid sides
    # log-uniform: mean of log n at the middle of [log 500, log 50000]
    assert abs(np.log(ns).mean() - 0.5 * (np.log(500) + np.log(50_000))) < 0.1
    assert 20.5e6 < ns.sum() < 23.5e6  # about 2048 x 10 749 rows
    for A, b in sy[:8]:
        check_csr(A)
        assert len(b) == len(A[0]) - 1


def test_rhs_and_seeds():
    A = I.convdiff3d(12, eps=(0.1, 0.1, 0.1), seed=3)
    b = I.rhs_ones_noise(A, 1e-3, 5)
    a1 = np.bincount(rows_of(A), weights=A[2])  # A 1
    assert abs((b - a1).std() - 1e-3) < 1e-4 and abs((b - a1).mean()) < 2e-4
    assert np.array_equal(b, I.rhs_ones_noise(A, 1e-3, 5))
    assert not np.array_equal(b, I.rhs_ones_noise(A, 1e-3, 6))
    P1, P2 = I.powerlaw_random(2000, seed=8), I.powerlaw_random(2000, seed=8)
    assert all(np.array_equal(x, y) for x, y in zip(P1, P2))
    P3 = I.powerlaw_random(2000, seed=9)
    assert not (len(P3[1]) == len(P1[1]) and np.array_equal(P3[1], P1[1]))
    B1 = I.convdiff3d(8, eps=(0.1, 0.1, 0.1), seed=1)
    B2 = I.convdiff3d(8, eps=(0.1, 0.1, 0.1), seed=2)
    assert np.array_equal(B1[1], B2[1]) and not np.array_equal(B1[2], B2[2])  # velocities

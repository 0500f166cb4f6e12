"""Seeded synthetic workloads for the GMRES solver (inputs only).

The paper measures on SuiteSparse matrices with solutions drawn from U(0, 1)
(Sec. 4).  Those matrices are not available here, so these generators build
matrices of the same kind -- sparse, non-symmetric, from convection-diffusion
discretisations and from a random power-law pattern -- at the sizes of the
benchmarked workloads.  Right-hand sides are ``b = A 1 + N(0, sigma^2)``.

This module holds no step of the solver.  Both the CUDA tests and the CPU
oracle tests draw their inputs from it; it imports neither side.

Matrices are returned as ``(rowptr int32[n+1], colind int32[nnz],
vals float64[nnz])`` with column indices sorted inside each row.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "convdiff2d", "convdiff3d", "powerlaw_random", "rhs_ones_noise", "batched_convdiff2d",
    "random_dd", "WORKLOADS", "workload",
]


def _stencil_csr(shape, eps, vel):
    """First-order upwind convection-diffusion on a structured grid.

    Discretises ``-sum_a eps_a d2u/dx_a^2 + v . grad u`` on the unit square/cube
    with h = 1/(N_a + 1) per axis (taken equal: h from the first axis) and
    homogeneous Dirichlet boundaries; every row is multiplied by h^2/eps_0 so
    that the diffusion weight of axis a is d_a = eps_a/eps_0 and the convection
    weight is c_a = h v_a / eps_0.  Row entries: centre sum_a (2 d_a + |c_a|),
    lower neighbour along a  -d_a - max(c_a, 0), upper  -d_a - max(-c_a, 0).
    ``vel`` has shape (n, dim)."""
    dims = len(shape)
    n = int(np.prod(shape))
    h = 1.0 / (shape[0] + 1)
    eps = np.asarray(eps, dtype=np.float64)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    stride = 1
    strides = []
    rem = idx
    for a in range(dims):
        coords.append(rem % shape[a])
        rem = rem // shape[a]
        strides.append(stride)
        stride *= shape[a]
    # entries per row: up to 2*dims neighbours + centre, emitted in column order
    cols = []
    vals = []
    valid = []
    diag = np.zeros(n)
    lower = []
    upper = []
    for a in range(dims):
        d = eps[a] / eps[0]
        c = h * vel[:, a] / eps[0]
        diag += 2.0 * d + np.abs(c)
        lower.append(-d - np.maximum(c, 0.0))
        upper.append(-d - np.maximum(-c, 0.0))
    # column order: lower neighbours from the largest stride down, centre,
    # upper neighbours from the smallest stride up -> ascending column index
    for a in reversed(range(dims)):
        cols.append(idx - strides[a])
        vals.append(lower[a])
        valid.append(coords[a] > 0)
    cols.append(idx)
    vals.append(diag)
    valid.append(np.ones(n, dtype=bool))
    for a in range(dims):
        cols.append(idx + strides[a])
        vals.append(upper[a])
        valid.append(coords[a] < shape[a] - 1)
    C = np.stack(cols, axis=1)
    Vv = np.stack(vals, axis=1)
    M = np.stack(valid, axis=1)
    counts = M.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = C[M].astype(np.int32)
    values = Vv[M].astype(np.float64)
    return rowptr.astype(np.int32), colind, values


class StencilFamily3D:
    """Matrices of the 3-D 7-point upwind family on one N^3 grid.

    The sparsity pattern (and the order of the entries) is fixed by the grid,
    so it is built once; ``values(eps, seed)`` returns only the value array of
    the matrix ``convdiff3d(N, eps, seed)`` would build (same entries, same
    order)."""

    def __init__(self, N):
        self.N = N
        n = N ** 3
        self.n = n
        idx = np.arange(n, dtype=np.int64)
        self.coords = [idx % N, (idx // N) % N, idx // (N * N)]
        self.strides = [1, N, N * N]
        valid = []
        for a in reversed(range(3)):
            valid.append(self.coords[a] > 0)
        valid.append(np.ones(n, dtype=bool))
        for a in range(3):
            valid.append(self.coords[a] < N - 1)
        self.mask = np.stack(valid, axis=1)
        A = convdiff3d(N, seed=0)
        self.rowptr, self.colind = A[0], A[1]

    def values(self, eps, seed):
        N = self.N
        n = self.n
        h = 1.0 / (N + 1)
        v = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, 3))
        eps = np.asarray(eps, dtype=np.float64)
        diag = np.zeros(n)
        lower, upper = [], []
        for a in range(3):
            d = eps[a] / eps[0]
            c = h * v[:, a] / eps[0]
            diag += 2.0 * d + np.abs(c)
            lower.append(-d - np.maximum(c, 0.0))
            upper.append(-d - np.maximum(-c, 0.0))
        vals = [lower[a] for a in reversed(range(3))] + [diag] + upper
        return np.stack(vals, axis=1)[self.mask].astype(np.float64)

    def matrix(self, eps, seed):
        return self.rowptr, self.colind, self.values(eps, seed)


def convdiff2d(nx, ny=None, pe=10.0, vel=None, seed=0):
    """2-D 5-point upwind convection-diffusion, eps = 1/pe on both axes.

    ``vel`` None -> constant v = (1, 1)/sqrt(2); ``"random"`` -> i.i.d.
    U[-1, 1]^2 per node from ``seed``."""
    ny = nx if ny is None else ny
    n = nx * ny
    if vel is None:
        v = np.tile(np.array([1.0, 1.0]) / math.sqrt(2.0), (n, 1))
    elif isinstance(vel, str) and vel == "random":
        v = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, 2))
    else:
        v = np.tile(np.asarray(vel, dtype=np.float64), (n, 1))
    e = 1.0 / pe
    return _stencil_csr((nx, ny), (e, e), v)


def convdiff3d(N, eps=(0.1, 0.1, 0.1), seed=0, vel="random"):
    """3-D 7-point upwind convection-diffusion on an N^3 grid.

    ``eps`` gives the per-axis diffusion (anisotropy 1:10:100 is
    ``(0.1, 1.0, 10.0)``); ``vel="random"`` draws v ~ U[-1, 1]^3 per node."""
    n = N ** 3
    if isinstance(vel, str) and vel == "random":
        v = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, 3))
    else:
        v = np.tile(np.asarray(vel, dtype=np.float64), (n, 1))
    return _stencil_csr((N, N, N), eps, v)


def _powerlaw_lengths(rng, n, lmin, lmax, alpha):
    L = np.arange(lmin, lmax + 1, dtype=np.float64)
    p = L ** (-alpha)
    p /= p.sum()
    cdf = np.cumsum(p)
    u = rng.random(n)
    return (lmin + np.searchsorted(cdf, u, side="right")).clip(lmin, lmax).astype(np.int64)


def powerlaw_random(n, lmin=3, lmax=200, alpha=1.734, dom=1.2, seed=0):
    """Random non-symmetric sparse matrix with power-law row lengths.

    Row length L (diagonal included) follows P(L) ~ L^-alpha on [lmin, lmax]
    (mean ~16 for the defaults); the L-1 off-diagonal columns are distinct,
    uniform over [0, n) without the diagonal, with N(0, 1) values; the
    diagonal is ``dom`` times the row's off-diagonal absolute sum."""
    rng = np.random.default_rng(seed)
    lmax = min(lmax, n)
    lmin = min(lmin, lmax)
    L = _powerlaw_lengths(rng, n, lmin, lmax, alpha)
    k = L - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    tot = int(k.sum())
    cols = rng.integers(0, n - 1, size=tot, dtype=np.int64)
    cols += cols >= rows  # skip the diagonal
    # make the columns of every row distinct: redraw duplicates until none remain
    for _ in range(256):
        order = np.lexsort((cols, rows))
        rows, cols = rows[order], cols[order]
        dup = np.zeros(tot, dtype=bool)
        dup[1:] = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        nd = int(dup.sum())
        if nd == 0:
            break
        c = rng.integers(0, n - 1, size=nd, dtype=np.int64)
        c += c >= rows[dup]
        cols[dup] = c
    else:  # pragma: no cover
        raise RuntimeError("could not draw distinct columns")
    offv = rng.standard_normal(tot)
    absrow = np.zeros(n)
    np.add.at(absrow, rows, np.abs(offv))
    diag = dom * absrow
    allr = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    allc = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    allv = np.concatenate([offv, diag])
    order = np.lexsort((allc, allr))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(allr, minlength=n), out=rowptr[1:])
    return rowptr.astype(np.int32), allc[order].astype(np.int32), allv[order]


def random_dd(n, density=0.2, dom=1.5, seed=0, nonsym=True):
    """Small dense-ish random diagonally dominant test matrix in CSR."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) * (rng.random((n, n)) < density)
    if not nonsym:
        A = A + A.T
    np.fill_diagonal(A, 0.0)
    np.fill_diagonal(A, dom * np.abs(A).sum(axis=1) + 1.0)
    return dense_to_csr(A)


def dense_to_csr(A):
    """CSR of the nonzeros of a dense array (diagonal always kept)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    mask = A != 0
    np.fill_diagonal(mask, True)
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    r, c = np.nonzero(mask)
    return rowptr.astype(np.int32), c.astype(np.int32), A[r, c].astype(np.float64)


def csr_to_dense(A):
    rowptr, colind, vals = A
    n = len(rowptr) - 1
    D = np.zeros((n, n))
    r = np.repeat(np.arange(n), np.diff(rowptr))
    D[r, colind] = vals
    return D


def rhs_ones_noise(A, sigma=1e-3, seed=0):
    """b = A 1 + N(0, sigma^2) noise (the row sums plus seeded noise)."""
    rowptr, colind, vals = A
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    b = np.bincount(rows, weights=vals, minlength=n)
    if sigma > 0:
        b = b + np.random.default_rng(seed).normal(0.0, sigma, size=n)
    return b


def batched_convdiff2d(count=2048, nmin=500, nmax=50000, pe_range=(1.0, 50.0), seed=0):
    """Independent 2-D convection-diffusion systems of uneven size.

    Sizes are log-uniform in [nmin, nmax]; grid nx = round(sqrt(n)),
    ny = round(n / nx); Peclet per system uniform in ``pe_range``; system i
    uses its own seed ``seed + i`` for the right-hand-side noise.  Returns a
    list of (A, b)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=count))
    pes = rng.uniform(pe_range[0], pe_range[1], size=count)
    out = []
    for i in range(count):
        nx = max(1, int(round(math.sqrt(ns[i]))))
        ny = max(1, int(round(ns[i] / nx)))
        A = convdiff2d(nx, ny, pe=float(pes[i]))
        out.append((A, rhs_ones_noise(A, 1e-3, seed + 1 + i)))
    return out


# Named workloads.  "full" entries are the benchmarked sizes, "small" entries
# are the same families at sizes the CPU oracle finishes in seconds.
WORKLOADS = {
    "convdiff2d_64": dict(kind="2d", N=64, pe=10.0, m=50, ortho="mgs", prec="fp64",
                          desc="2-D 5-point upwind convection-diffusion 64^2, Pe 10"),
    "convdiff3d_160": dict(kind="3d", N=160, eps=(0.1, 0.1, 0.1), m=100, ortho="cgsr",
                           prec="mixed",
                           desc="3-D 7-point upwind convection-diffusion 160^3, v~U[-1,1]^3"),
    "convdiff3d_24": dict(kind="3d", N=24, eps=(0.1, 0.1, 0.1), m=100, ortho="cgsr",
                          prec="mixed"),
    "convdiff3d_96": dict(kind="3d", N=96, eps=(0.1, 0.1, 0.1), m=100, ortho="cgsr",
                          prec="mixed"),
    "convdiff3d_160_ilu": dict(kind="3d", N=160, eps=(0.1, 0.1, 0.1), m=100, ortho="cgsr",
                               prec="mixed", precond="ilu",
                               desc="3-D convection-diffusion 160^3, ILU(0) left preconditioner"),
    "convdiff3d_96_ilu": dict(kind="3d", N=96, eps=(0.1, 0.1, 0.1), m=100, ortho="cgsr",
                              prec="mixed", precond="ilu",
                              desc="3-D convection-diffusion 96^3, ILU(0) left preconditioner"),
    "powerlaw_2m": dict(kind="powerlaw", n=2_000_000, m=50, ortho="mgs", prec="mixed_bf16",
                        desc="random power-law rows 3-200 (mean 16), diagonal 1.2 x row sum"),
    "powerlaw_20k": dict(kind="powerlaw", n=20_000, m=50, ortho="mgs", prec="mixed_bf16"),
    "aniso3d_128": dict(kind="3d", N=128, eps=(0.1, 1.0, 10.0), m=50, ortho="cgsr",
                        prec="mixed", precond="learned",
                        desc="3-D convection-diffusion 128^3, anisotropy 1:10:100, learned SpAI"),
    "aniso3d_24": dict(kind="3d", N=24, eps=(0.1, 1.0, 10.0), m=50, ortho="cgsr", prec="mixed",
                       precond="learned"),
}


def workload(name, seed=20110185):
    """(A, b, spec) for a named workload."""
    spec = WORKLOADS[name]
    if spec["kind"] == "2d":
        A = convdiff2d(spec["N"], pe=spec["pe"])
    elif spec["kind"] == "3d":
        A = convdiff3d(spec["N"], eps=spec["eps"], seed=seed)
    else:
        A = powerlaw_random(spec["n"], seed=seed)
    b = rhs_ones_noise(A, 1e-3, seed + 1)
    return A, b, spec

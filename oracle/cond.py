"""2-norm condition numbers of the convection-diffusion workloads.

TEST INFRASTRUCTURE ONLY: the full-size GPU tests bound the forward error of
a solution by kappa_2(A) times its relative residual (the standard bound
||x - x*|| / ||x*|| <= kappa_2(A) ||b - A x|| / ||b||), and the tolerance of
a comparison between two solutions is the sum of the two bounds.  kappa_2 of
the 160^3 matrix is too large a problem for a sparse factorisation, so it is
estimated on smaller grids of the same family and extrapolated in (N + 1)^2,
the growth of the condition number of a second-order difference operator with
mesh width h = 1 / (N + 1).

sigma_max comes from the power method on A^T A, sigma_min from inverse
iteration on A^T A with a sparse LU factorisation of A (scipy's SuperLU); on
small grids both agree with a dense SVD (a CPU test checks that).

    python -m oracle.cond     # writes tests/golden/convdiff3d_kappa.json
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(os.path.dirname(HERE), "tests", "golden")


def _scipy_csr(A):
    import scipy.sparse as sp

    rp, ci, va = A
    n = len(rp) - 1
    return sp.csr_matrix((np.asarray(va, np.float64), np.asarray(ci), np.asarray(rp)),
                         shape=(n, n))


def sigma_extremes(A, iters=300, seed=0, rtol=1e-9):
    """(sigma_min, sigma_max) of the CSR matrix A."""
    import scipy.sparse.linalg as sla

    S = _scipy_csr(A)
    n = S.shape[0]
    rng = np.random.default_rng(seed)
    # largest: power method on A^T A
    x = rng.standard_normal(n)
    x /= np.linalg.norm(x)
    smax = 0.0
    for _ in range(iters):
        y = S.T @ (S @ x)
        lam = np.linalg.norm(y)
        x = y / lam
        new = np.sqrt(lam)
        if abs(new - smax) <= rtol * new:
            smax = new
            break
        smax = new
    # smallest: inverse iteration on A^T A, (A^T A)^-1 = A^-1 A^-T
    lu = sla.splu(S.tocsc())
    x = rng.standard_normal(n)
    x /= np.linalg.norm(x)
    smin = np.inf
    for _ in range(iters):
        y = lu.solve(lu.solve(x, trans="T"))
        lam = np.linalg.norm(y)
        x = y / lam
        new = 1.0 / np.sqrt(lam)
        if abs(new - smin) <= rtol * new:
            smin = new
            break
        smin = new
    return smin, smax


def main():
    from paper_2011_01850_gb300 import inputs as I

    rows = []
    for N in (16, 24, 32, 40, 48):
        A = I.convdiff3d(N, eps=(0.1, 0.1, 0.1), seed=20110185)
        t = time.time()
        smin, smax = sigma_extremes(A)
        rows.append(dict(N=N, sigma_min=smin, sigma_max=smax, kappa=smax / smin,
                         seconds=round(time.time() - t, 1)))
        print(rows[-1], flush=True)
    # kappa = c (N + 1)^2: least squares in c over the three largest grids
    big = rows[-3:]
    h2 = np.array([(r["N"] + 1) ** 2 for r in big], float)
    kap = np.array([r["kappa"] for r in big])
    c = float(np.dot(h2, kap) / np.dot(h2, h2))
    out = dict(family="convdiff3d, eps = 0.1, v ~ U[-1,1]^3 per node (seed 20110185)",
               grids=rows, fit="kappa = c (N + 1)^2 over N = 32, 40, 48", c=c,
               kappa_96=c * 97 ** 2, kappa_160=c * 161 ** 2,
               command="python -m oracle.cond")
    with open(os.path.join(GOLDEN, "convdiff3d_kappa.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

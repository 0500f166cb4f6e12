"""The condition-number estimator the full-size tolerances use (CPU).

oracle/cond.py estimates sigma_min by inverse iteration on A^T A through a
sparse LU factorisation and sigma_max by the power method; on grids small
enough for a dense SVD both must agree with numpy's singular values, and the
stored estimates of the 3-D family must grow like (N + 1)^2.
"""
import json
import os

import numpy as np

from oracle import cond as C
from paper_2011_01850_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_sigma_extremes_match_dense_svd():
    for N in (5, 8):
        A = I.convdiff3d(N, eps=(0.1, 0.1, 0.1), seed=20110185)
        smin, smax = C.sigma_extremes(A, iters=2000, rtol=1e-13)
        sv = np.linalg.svd(I.csr_to_dense(A), compute_uv=False)
        assert abs(smax - sv[0]) <= 1e-8 * sv[0], (N, smax, sv[0])
        assert abs(smin - sv[-1]) <= 1e-8 * sv[-1], (N, smin, sv[-1])


def test_stored_kappa_follows_mesh_law():
    with open(os.path.join(GOLDEN, "convdiff3d_kappa.json")) as f:
        k = json.load(f)
    for r in k["grids"]:
        c = r["kappa"] / (r["N"] + 1) ** 2
        assert abs(c - k["c"]) <= 0.1 * k["c"], r
    assert abs(k["kappa_160"] - k["c"] * 161 ** 2) <= 1e-9 * k["kappa_160"]

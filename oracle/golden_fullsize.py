"""Stored oracle results for the 160^3 mixed CGSR GMRES(100) workload.

TEST INFRASTRUCTURE ONLY: this script calls nothing but the CPU oracle (the
single-threaded parity build of gmres_oracle.c) and the seeded input
generators, and writes the expected values the full-size GPU tests compare
against.  Nothing here comes from the CUDA library.

Parts (each its own command, so they can run side by side; every part takes
tens of minutes on one core):

    python -m oracle.golden_fullsize schedule   # mixed solve, tol 1e-10
    python -m oracle.golden_fullsize solution   # binary64 solve, tol 1e-13

``schedule`` runs the oracle's fully mixed solver (Sec. 4: binary64 residual
and update, binary32 cycle; tau = 1e-6 for the first cycle, later cycles as
long as the first) to the workload's target and writes its restart schedule
and the binary64 relative residual after every cycle to
tests/golden/convdiff3d_160_schedule.json.

``solution`` runs the oracle's binary64 solver to tol 1e-13, so that its x is
within kappa * 1e-13 of the exact solution, and writes x at 65 536 seeded
indices (and the indices) to tests/golden/convdiff3d_160_x.npz.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(os.path.dirname(HERE), "tests", "golden")
NAME = "convdiff3d_160"
SEED = 20110185
NSAMPLE = 65536
SAMPLE_SEED = 160


def sample_indices(n):
    """Sorted distinct row indices of the stored solution entries."""
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(n, NSAMPLE, replace=False)).astype(np.int32)


def schedule():
    import oracle as O
    from paper_2011_01850_gb300 import inputs as I

    A, b, spec = I.workload(NAME, seed=SEED)
    t = time.time()
    _, info = O.gmres(A, b, m=spec["m"], tol=1e-10, ortho=O.CGSR, prec=O.MIXED,
                      maxiter=100000, history=True)
    out = dict(workload=NAME, seed=SEED, m=spec["m"], ortho="cgsr", prec="mixed", tol=1e-10,
               tau=O.default_tau(O.MIXED), repeat_first=True, iters=info["iters"],
               restarts=info["restarts"], first_len=info["first_len"],
               converged=info["converged"], relres=info["relres"],
               cycle_relres=[float(v) for v in info["cycle_relres"]],
               oracle_seconds=round(time.time() - t, 1),
               command="python -m oracle.golden_fullsize schedule")
    path = os.path.join(GOLDEN, NAME + "_schedule.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out), flush=True)


def solution():
    import oracle as O
    from paper_2011_01850_gb300 import inputs as I

    A, b, spec = I.workload(NAME, seed=SEED)
    n = len(b)
    t = time.time()
    x, info = O.gmres(A, b, m=spec["m"], tol=1e-13, ortho=O.CGSR, prec=O.FP64,
                      maxiter=100000)
    secs = round(time.time() - t, 1)
    idx = sample_indices(n)
    meta = dict(workload=NAME, seed=SEED, m=spec["m"], ortho="cgsr", prec="fp64", tol=1e-13,
                iters=info["iters"], restarts=info["restarts"], relres=info["relres"],
                converged=info["converged"], oracle_seconds=secs, n=n,
                xnorm=float(np.linalg.norm(x)),
                command="python -m oracle.golden_fullsize solution")
    path = os.path.join(GOLDEN, NAME + "_x.npz")
    np.savez_compressed(path, idx=idx, x=x[idx], meta=json.dumps(meta))
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    {"schedule": schedule, "solution": solution}[sys.argv[1]]()

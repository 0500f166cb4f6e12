"""Training driver and helpers for the learned SpAI right preconditioner.

Every arithmetic step -- features, the MLP forward and backward passes, the
SpMVs with M, A and A^T, the loss, Adam -- runs in the library's CUDA kernels
(gmres_spai_* in include/gmres_gb300.h).  This module only orders those calls:
it walks a stream of training matrices of one sparsity pattern (refreshing the
values of a single handle with gmres_set_values), optionally adds residual
vectors that short unpreconditioned solves of the training systems leave
behind as extra probes, and keeps the parameters and Adam moments on the
device.

Initialisation: the Jacobi parameters (the network outputs [p == q], so
M = D^-1) plus N(0, 0.02^2) noise; Adam with lr 3e-3 and 8 Rademacher probes
per step learn M's values from there.
"""
from __future__ import annotations

import math

import numpy as np

from . import gmres as G
from . import inputs as I

NPARAM = G.SPAI_NPARAM


def jacobi_params():
    """Parameters whose network outputs exactly [p == q] (M = D^-1)."""
    p = np.zeros(NPARAM, dtype=np.float32)
    p[0 * 8 + 2] = 1.0          # W1[0][2]: the [p == q] feature into unit 0
    p[576 + 0] = 1.0            # W2[0][0]
    p[576 + 4096 + 64 + 0] = 1.0  # w3[0]
    return p


def init_params(seed=0, noise=0.02):
    rng = np.random.default_rng(seed)
    return (jacobi_params() + noise * rng.standard_normal(NPARAM)).astype(np.float32)


_FAMILIES = {}


def training_matrix(N, index, seed=20110185):
    """Training system `index` of the 3-D family: 7-point upwind
    convection-diffusion on N^3, v ~ U[-1, 1]^3 per node, diffusion
    0.1 * (1, r1, r2) with r1, r2 log-uniform in [1, 100]."""
    if N not in _FAMILIES:
        _FAMILIES[N] = I.StencilFamily3D(N)
    fam = _FAMILIES[N]
    rng = np.random.default_rng(seed + 7919 * (index + 1))
    r = np.exp(rng.uniform(0.0, math.log(100.0), size=2))
    A = fam.matrix((0.1, 0.1 * r[0], 0.1 * r[1]), seed + index)
    b = I.rhs_ones_noise(A, 1e-3, seed + 100000 + index)
    return A, b


class Trainer:
    """Owns one handle (the training pattern) and the device-side state."""

    def __init__(self, A0, params=None, stream=None):
        import torch
        self.torch = torch
        self.solver = G.Solver(A0, flags=G.CREATE_TRANSPOSE, stream=stream)
        self.n = self.solver.n
        p = init_params() if params is None else np.asarray(params, np.float32)
        self.params = torch.tensor(p, device="cuda")
        self.m = torch.zeros(NPARAM, device="cuda")
        self.v = torch.zeros(NPARAM, device="cuda")
        self.step = 0
        self.history = []

    def solver_probes(self, b, counts=(5, 15)):
        """Residuals b - A x of short unpreconditioned mixed solves (x after
        `c` inner iterations for each c in counts), scaled to unit RMS."""
        torch = self.torch
        h = self.solver.h
        o = G.gmres_get_opts(h)
        o.precond = 0
        G.gmres_set_opts(h, o)
        db = torch.tensor(b, device="cuda", dtype=torch.float64)
        out = torch.empty((len(counts), self.n), device="cuda", dtype=torch.float32)
        z = torch.empty(self.n, device="cuda", dtype=torch.float64)
        for i, c in enumerate(counts):
            x = torch.zeros(self.n, device="cuda", dtype=torch.float64)
            G.gmres_solve(h, db, x, 30, 1e-12, G.ORTHO_CGSR, G.MIXED, int(c))
            nrm = G.gmres_residual(h, db, x, z)
            out[i] = (z * (math.sqrt(self.n) / max(nrm, 1e-300))).float()
        return out.contiguous()

    def train_on(self, A=None, b=None, steps=1, nprobe=8, lr=3e-3, seed=1, use_solver=False):
        """`steps` Adam steps on matrix A (None: the handle's current one)."""
        if A is not None:
            G.gmres_set_values(self.solver.h, np.ascontiguousarray(A[2], np.float64))
        Zx = self.solver_probes(b) if (use_solver and b is not None) else None
        for _ in range(steps):
            self.step += 1
            loss = G.gmres_spai_train_step(
                self.solver.h, self.params, self.m, self.v, self.step, nprobe,
                seed * 1000003 + self.step, Zx, 0 if Zx is None else Zx.shape[0], lr)
            self.history.append(loss)
        return self.history[-1]

    def params_host(self):
        return self.params.detach().cpu().numpy().copy()

    def close(self):
        self.solver.close()


def train(N=64, count=2000, steps_per_matrix=1, nprobe=8, lr=3e-3, solver_every=10, seed=1,
          stream=None, log=None):
    """Train on `count` seeded matrices of the 3-D family at N^3; returns
    (params, loss history)."""
    A0, b0 = training_matrix(N, 0)
    tr = Trainer(A0, stream=stream)
    try:
        for i in range(count):
            A, b = training_matrix(N, i)
            tr.train_on(A, b, steps=steps_per_matrix, nprobe=nprobe, lr=lr, seed=seed,
                        use_solver=(solver_every > 0 and i % solver_every == 0))
            if log is not None and (i + 1) % max(1, count // 20) == 0:
                log("matrix %d/%d loss %.4e" % (i + 1, count, tr.history[-1]))
        return tr.params_host(), list(tr.history)
    finally:
        tr.close()


if __name__ == "__main__":  # pragma: no cover - offline training entry point
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(description="train the learned SpAI preconditioner")
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--record", default=None,
                    help="write the run's settings, wall time and loss history (JSON)")
    args = ap.parse_args()
    t0 = time.time()
    p, hist = train(N=args.N, count=args.count, log=print)
    secs = time.time() - t0
    print(json.dumps({"seconds": secs, "first_loss": hist[0],
                      "last_loss": float(np.mean(hist[-20:]))}))
    if args.out:
        np.save(args.out, p)
    if args.record:
        import sys
        rec = {"command": "python -m paper_2011_01850_gb300.spai " + " ".join(sys.argv[1:]),
               "seconds": round(secs, 1), "matrices": args.count, "grid": args.N,
               "family": "3-D 7-point upwind convection-diffusion, v ~ U[-1,1]^3 per node, "
                         "diffusion 0.1 (1, r1, r2), r1, r2 log-uniform in [1, 100]",
               "adam": {"lr": 3e-3, "beta1": 0.9, "beta2": 0.999, "eps": 1e-8},
               "init": "Jacobi parameters + N(0, 0.02^2), seed 0",
               "probes": "8 Rademacher probes per step (counter-based, seed 1000003 s + step); "
                         "every 10th matrix also the residuals of unpreconditioned mixed "
                         "CGSR GMRES(30) after 5 and 15 inner iterations (unit RMS)",
               "steps": len(hist), "loss": [float(v) for v in hist]}
        with open(args.record, "w") as f:
            json.dump(rec, f)
            f.write("\n")

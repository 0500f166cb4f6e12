"""Element-wise parity at the benchmarked sizes (marker: gpu).

* One inner iteration replayed from the oracle's own basis on the 96^3
  convection-diffusion matrix (n = 884 736, several 512-row slices per
  block), for basis sizes 1, 16, 32, 64, 96 and 100: the binary32 pass-B
  kernel instantiations for 2, 4, 8, 12 and 17 vectors per warp, and the
  cooperative MGS kernel.  The GPU's Hessenberg column, h_{j+1,j} and
  v_{j+1} are compared entry by entry with the oracle's binary64 evaluation
  of the same iteration on the same stored operands (A rounded as the GPU
  holds it, the basis as stored), within a running error bound of the GPU's
  arithmetic (see _step_bound).
* A whole restart cycle of 100 inner iterations at 96^3 in MIXED and
  MIXED_FP16 against the oracle's cycle in the same precision.
* The tau restart rule (Sec. 3, second strategy; the first cycle of every
  mixed solve) on the GPU: the cycle ends at the first iteration whose own
  |s_{j+1}| <= tau * beta, and the solver's first cycle has the oracle's
  length within one iteration.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G

U32, U64 = 2.0 ** -24, 2.0 ** -53
# unit roundoff of each basis storage format (round to nearest)
STORE_U = {O.FP64: 0.0, O.MIXED: U32, O.MIXED_BF16: 2.0 ** -8, O.MIXED_FP16: 2.0 ** -11}
O2G = {O.FP64: 0, O.MIXED: 1, O.MIXED_BF16: 2, O.MIXED_FP16: 3}
# Upper bound on the number of additions a product passes through in any GPU
# reduction (per-thread partial over its slices, warp butterfly, block, the
# column reduction over blocks, the block-ordered exchange of cooperative MGS):
# under 200 at 96^3 and 160^3.
GPU_DEPTH = 512


def _fp16_scale(n):
    """The binary16 basis scale 2^floor(log2(n)/2)."""
    return 2.0 ** (int(math.floor(math.log2(n))) // 2)


def gamma(k, u):
    return k * u / (1.0 - k * u)


def _step_bound(A_used, V, ortho, u, depth):
    """First-order error bound of one inner iteration computed with unit
    roundoff u and reductions of at most `depth` additions, against the exact
    iteration on the same operands (Higham, Accuracy and Stability of
    Numerical Algorithms, Sec. 3.1: a k-term sum or inner product in any
    order is within gamma_k = k u / (1 - k u) of the exact one relative to
    the sum of absolute values).  Errors are tracked entry by entry (E) and
    in the 2-norm (eps); the projections I - V^T V of Gram-Schmidt do not
    grow the 2-norm of an error already in w.  Returns (h_exact, hn_exact,
    v_exact, bound_h, bound_hn, bound_v); h has j entries."""
    rp, ci, va = A_used
    n = len(rp) - 1
    j = V.shape[0]
    rows = np.repeat(np.arange(n), np.diff(rp))
    vj = V[-1]
    w = np.zeros(n)
    np.add.at(w, rows, va * vj[ci])
    aw = np.zeros(n)
    np.add.at(aw, rows, np.abs(va) * np.abs(vj[ci]))
    kmax = int(np.diff(rp).max())
    E = gamma(kmax, u) * aw          # entry-wise bound of the error in w = A v_j
    eps = np.linalg.norm(E)          # its 2-norm
    aV = np.abs(V)
    gd = gamma(depth, u)
    h = np.zeros(j)
    dh = np.zeros(j)
    if ortho == O.CGSR:
        gj = gamma(j + 1, u)
        for _ in range(2):
            g = V @ w
            rnd = gd * (aV @ np.abs(w))                 # rounding of the inner products
            dg = np.minimum(aV @ E, eps) + rnd          # + the error already in w
            rho = gj * (np.abs(w) + aV.T @ np.abs(g))   # rounding of w - V^T g
            E = E + aV.T @ dg + rho
            eps = eps + np.linalg.norm(rnd) + np.linalg.norm(rho)
            w = w - V.T @ g
            h += g
            dh += dg
        dh += u * np.abs(h)
    else:
        for i in range(j):
            hi = V[i] @ w
            rnd = gd * (aV[i] @ np.abs(w))
            dh[i] = min(aV[i] @ E, eps) + rnd
            rho = 2 * u * (np.abs(w) + abs(hi) * aV[i])
            E = E + aV[i] * dh[i] + rho
            eps = eps + rnd + np.linalg.norm(rho)
            w = w - hi * V[i]
            h[i] = hi
    hn = np.linalg.norm(w)
    dhn = eps + gamma(depth + 2, u) * hn
    v = w / hn
    dv = E / hn + np.abs(v) * dhn / hn + u * np.abs(v)
    return h, hn, v, dh, dhn, dv


@pytest.fixture(scope="module")
def cd96():
    A, b, spec = I.workload("convdiff3d_96", seed=20110185)
    return A, b


_cycles = {}


def oracle_cycle96(A, b, prec, ortho):
    key = (prec, ortho)
    if key not in _cycles:
        _cycles.clear()  # one basis (101 x 884 736 doubles) at a time
        _cycles[key] = O.arnoldi_cycle(A, b, 100, ortho=ortho, prec=prec, kmax=100)
    return _cycles[key]


STEP_CASES = [(O.MIXED, O.CGSR), (O.MIXED_FP16, O.CGSR), (O.FP64, O.CGSR), (O.MIXED, O.MGS)]


@pytest.mark.parametrize("prec,ortho", STEP_CASES,
                         ids=["mixed-cgsr", "fp16-cgsr", "fp64-cgsr", "mixed-mgs"])
def test_step_replay_96(cd96, prec, ortho, gpulib):
    A, b = cd96
    rp, ci, va = A
    n = len(b)
    cyc = oracle_cycle96(A, b, prec, ortho)
    assert cyc["j"] == 100
    # the operands as the GPU holds them: A's binary32 copy for the binary32
    # cycle, the basis exactly as the oracle stored it
    A_used = (rp, ci, va if prec == O.FP64 else va.astype(np.float32).astype(np.float64))
    u = U64 if prec == O.FP64 else U32
    s = G.Solver(A, stream=torch.cuda.current_stream())
    worst = 0.0
    for ncols in (1, 16, 32, 64, 96, 100):
        V = cyc["V"][:ncols]
        hg, vg = G.gmres_arnoldi_step(s.h, V, ortho, O2G[prec])
        # the oracle's binary64 evaluation of the same iteration
        ho, vo = O.arnoldi_step(A_used, V, ortho=ortho, prec=O.FP64)
        h, hn, v, dh, dhn, dv = _step_bound(A_used, V, ortho, u, GPU_DEPTH)
        # the oracle's own (sequential, binary64) error on top of the GPU's
        _, _, _, dho, dhno, dvo = _step_bound(A_used, V, ortho, U64, n)
        bh = 1.01 * (dh + dho) + 1e-300
        bhn = 1.01 * (dhn + dhno)
        # storage rounding: relative in the normal range; binary16 entries
        # below 2^-14 (after the power-of-two scale) are subnormal, spacing
        # 2^-24, so half of that, unscaled, bounds their absolute error
        sub = 2.0 ** -25 / _fp16_scale(n) if prec == O.MIXED_FP16 else 0.0
        bv = 1.01 * (dv + dvo) + STORE_U[prec] * np.abs(vo) + sub + 1e-300
        eh = np.abs(hg[:ncols] - ho[:ncols])
        assert np.all(eh <= bh), (ncols, float((eh / bh).max()))
        assert abs(hg[ncols] - ho[ncols]) <= bhn, (ncols, hg[ncols], ho[ncols], bhn)
        ev = np.abs(vg - vo)
        assert np.all(ev <= bv), (ncols, float((ev / bv).max()))
        # the GPU's binary32 result is a genuinely binary32 computation: no
        # closer to binary64 than its own rounding allows, and the bound is
        # not vacuous (the exact values are orders of magnitude above it)
        assert bh.max() < 1e-2 * max(np.abs(ho[:ncols]).max(), ho[ncols])
        worst = max(worst, float((eh / bh).max()), float((ev / bv).max()))
    s.close()
    print("worst error / bound:", worst)


def _cycle_tol(prec, n):
    """Tolerance of a whole restart cycle against the oracle's cycle in the
    same precision.  The oracle sums sequentially (error up to n u per inner
    product, about sqrt(n) u in practice), the GPU in trees; with
    probability above 1 - 1e-7 a sequential binary32 inner product of n terms
    is within 8 sqrt(n) u of the exact one (Higham and Mary's probabilistic
    bound), and later Arnoldi quantities inherit these per-step differences,
    so the bound is the two sides' 8 sqrt(n) u each, doubled for the
    propagation over the cycle, or the per-precision small-size tolerance
    (the 16-bit storage roundoff dominates those)."""
    base = {O.MIXED: 2e-4, O.MIXED_FP16: 2e-2, O.MIXED_BF16: 5e-2}[prec]
    return max(base, 32.0 * math.sqrt(n) * U32)


@pytest.mark.parametrize("prec", [O.MIXED, O.MIXED_FP16], ids=["mixed", "fp16"])
def test_cycle_parity_96(cd96, prec, gpulib):
    A, b = cd96
    n = len(b)
    m = 100
    o = oracle_cycle96(A, b, prec, O.CGSR)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    g = G.gmres_arnoldi(s.h, torch.tensor(b, device="cuda", dtype=torch.float64), m, m,
                        O.CGSR, O2G[prec], n=n)
    s.close()
    assert g["j"] == o["j"] == m
    tol = _cycle_tol(prec, n)
    beta = np.linalg.norm(b)

    def close(a, b_, scale, what):
        err = np.abs(a - b_).max() / scale
        assert err <= tol, (what, err, tol)
        return err

    j = m
    close(g["Hbar"][: j + 1, :j], o["Hbar"][: j + 1, :j], np.abs(o["Hbar"]).max(), "Hbar")
    close(g["H"][: j + 1, :j], o["H"][: j + 1, :j], np.abs(o["H"]).max(), "H")
    close(g["cs"][:j], o["cs"][:j], 1.0, "cs")
    close(g["sn"][:j], o["sn"][:j], 1.0, "sn")
    close(g["s"][: j + 1], o["s"][: j + 1], beta, "s")
    close(g["arn"][:j], o["arn"][:j], beta, "arn")
    close(g["y"][:j], o["y"][:j], np.abs(o["y"][:j]).max(), "y")
    close(g["u"], o["u"], np.abs(o["u"]).max(), "u")
    for k in range(0, j, 9):
        close(g["V"][k], o["V"][k], np.abs(o["V"][k]).max(), "V%d" % k)


def test_tau_rule_on_gpu(gpulib):
    """The first-cycle restart test (Sec. 3, second strategy; tau = 1e-6 as
    in Sec. 4.2): a cycle ends at the first inner iteration whose Arnoldi
    residual |s_{j+1}| is at most tau * beta, judged on the GPU's own
    residual history; the solver's first cycle is as long as the oracle's to
    within one iteration (the two sum in different orders, so a crossing
    within a rounding of tau * beta may land one iteration apart)."""
    A = I.convdiff3d(40, seed=3)
    b = I.rhs_ones_noise(A, 1e-3, 7)
    n = len(b)
    tau = 1e-6
    s = G.Solver(A, stream=torch.cuda.current_stream())
    s.set_opts(path=G.PATH_GRID)
    g = G.gmres_arnoldi(s.h, torch.tensor(b, device="cuda", dtype=torch.float64), 128, 128,
                        O.CGSR, G.MIXED, tau=tau, n=n)
    full = G.gmres_arnoldi(s.h, torch.tensor(b, device="cuda", dtype=torch.float64), 128, 128,
                           O.CGSR, G.MIXED, tau=0.0, n=n)
    # beta of the binary32 cycle: ||fl32(r0)|| (the GPU's value agrees to a
    # few binary32 roundings; the margin below covers that)
    beta = float(np.linalg.norm(b.astype(np.float32).astype(np.float64)))
    arn = full["arn"][: full["j"]]
    first = int(np.argmax(arn <= tau * beta)) + 1
    assert arn[first - 1] <= tau * beta * (1 + 1e-5)
    assert np.all(arn[: first - 1] > tau * beta * (1 - 1e-5))
    assert 1 < first < full["j"], (first, full["j"])
    assert g["j"] == first, (g["j"], first)
    np.testing.assert_array_equal(g["arn"][: g["j"]], full["arn"][: g["j"]])
    # the whole solver: first cycle as long as the oracle's (+-1)
    db = torch.tensor(b, device="cuda", dtype=torch.float64)
    dx = torch.zeros(n, device="cuda", dtype=torch.float64)
    _, st, info = s.solve(db, dx, m=128, tol=1e-10, ortho="cgsr", prec="mixed", maxiter=20000)
    s.close()
    assert st == G.OK
    _, oi = O.gmres(A, b, m=128, tol=1e-10, ortho=O.CGSR, prec=O.MIXED, maxiter=20000)
    assert abs(info["first_len"] - oi["first_len"]) <= 1, (info["first_len"], oi["first_len"])
    assert info["first_len"] == first

"""Pins for the CPU oracle: facts fixed by the paper and by the mathematics.

Every ``pin_*`` function checks the oracle against something other than itself
-- a library routine (LAPACK solve/lstsq through numpy, torch's bfloat16 and
numpy's binary16 conversions), a closed form, a hand-worked example, an
invariant of exact arithmetic, or brute force on a tiny input.  They are run
once against the real oracle (test_oracle_pins.py) and again against builds
with planted mistakes, each of which at least one pin must reject.
"""
from __future__ import annotations

import math
import os

import numpy as np

import oracle as O
from paper_2011_01850_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def _dense(A):
    return I.csr_to_dense(A)


# ---------------------------------------------------------------------------
# whole solver
# ---------------------------------------------------------------------------

def pin_lu_fp64():
    """Binary64 GMRES equals a dense LU solve (numpy/LAPACK) up to kappa*1e-13
    on random diagonally dominant non-symmetric systems (MGS and CGSR)."""
    for seed in range(3):
        A = I.random_dd(40, density=0.3, dom=0.6, seed=seed)
        D = _dense(A)
        b = np.random.default_rng(100 + seed).standard_normal(40)
        xl = np.linalg.solve(D, b)
        kappa = np.linalg.cond(D)
        for ortho in (O.MGS, O.CGSR):
            x, info = O.gmres(A, b, m=15, tol=1e-13, ortho=ortho, prec=O.FP64, maxiter=2000)
            err = np.linalg.norm(x - xl) / np.linalg.norm(xl)
            assert info["converged"], info
            assert err <= kappa * 1e-13, (seed, ortho, err, kappa)


def pin_exact_convergence():
    """Without restarts (m >= n) GMRES solves an n x n system in at most n steps."""
    n = 24
    rng = np.random.default_rng(7)
    D = rng.standard_normal((n, n)) + 6.0 * np.eye(n)
    A = I.dense_to_csr(D)
    b = rng.standard_normal(n)
    for ortho in (O.MGS, O.CGSR):
        x, info = O.gmres(A, b, m=n, tol=1e-12, ortho=ortho, prec=O.FP64, maxiter=n,
                          inner_factor=0.5)
        assert info["iters"] <= n and info["restarts"] == 1, info
        assert np.linalg.norm(b - D @ x) <= 1e-12 * np.linalg.norm(b), info


def pin_identity():
    """A = I: every cycle takes one inner iteration (w = v_1 breaks down at
    once); in binary64 one cycle gives x = b, while the binary32 correction of
    the mixed solver leaves an O(u32) error that the next one-step cycles
    remove."""
    n = 17
    A = I.dense_to_csr(np.eye(n))
    b = np.arange(1.0, n + 1)
    for ortho in (O.MGS, O.CGSR):
        x, info = O.gmres(A, b, m=10, tol=1e-10, ortho=ortho, prec=O.FP64, maxiter=50)
        assert info["iters"] == 1 and info["restarts"] == 1, info
        assert np.allclose(x, b, rtol=1e-14, atol=0), x
        x, info = O.gmres(A, b, m=10, tol=1e-10, ortho=ortho, prec=O.MIXED, maxiter=50)
        assert info["converged"] and info["iters"] == info["restarts"] <= 3, info
        assert np.allclose(x, b, rtol=1e-10, atol=0), x


def pin_diag_distinct():
    """A diagonal matrix with k distinct eigenvalues: the Krylov space of any b
    has dimension <= k, so GMRES ends (breakdown) after k steps with the exact
    solution."""
    k = 5
    vals = np.array([1.0, 2.0, 3.5, 7.0, 11.0])
    d = np.repeat(vals, 8)
    n = d.size
    A = I.dense_to_csr(np.diag(d))
    b = np.random.default_rng(3).uniform(0.5, 1.5, n)
    for ortho in (O.MGS, O.CGSR):
        x, info = O.gmres(A, b, m=20, tol=1e-12, ortho=ortho, prec=O.FP64, maxiter=100)
        assert info["iters"] == k, info
        assert np.allclose(x, b / d, rtol=1e-12, atol=0)


def pin_cyclic_shift():
    """Cyclic shift P e_i = e_{i+1}, b = e_1, x0 = 0: the Krylov vectors are
    e_1, e_2, ..., so the residual stays 1 for n-1 steps (complete stagnation)
    and the exact solution x = e_n appears at step n."""
    n = 12
    P = np.zeros((n, n))
    for i in range(n):
        P[(i + 1) % n, i] = 1.0
    A = I.dense_to_csr(P)
    b = np.zeros(n)
    b[0] = 1.0
    for ortho in (O.MGS, O.CGSR):
        cyc = O.arnoldi_cycle(A, b, m=n, ortho=ortho, prec=O.FP64)
        assert cyc["j"] == n, cyc["j"]
        assert np.allclose(cyc["arn"][: n - 1], 1.0, atol=1e-14)
        assert abs(cyc["arn"][n - 1]) <= 1e-14
        e_n = np.zeros(n)
        e_n[-1] = 1.0
        assert np.allclose(cyc["u"], e_n, atol=1e-13)


def pin_hand_2x2():
    """Every quantity of the hand-worked 2x2 cycle in tests/golden."""
    g = {}
    with open(os.path.join(HERE, "golden", "gmres_2x2_by_hand.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(None, 1)
            g[k] = float(eval(v, {"sqrt": math.sqrt}))
    A = I.dense_to_csr(np.array([[2.0, 1.0], [0.0, 1.0]]))
    b = np.array([1.0, 1.0])
    c = O.arnoldi_cycle(A, b, m=2, ortho=O.MGS, prec=O.FP64)
    tol = 1e-14
    assert c["j"] == g["iterations"]
    Hb = c["Hbar"]
    assert abs(Hb[0, 0] - g["hbar_1_1"]) < tol and abs(Hb[1, 0] - g["hbar_2_1"]) < tol
    assert abs(Hb[0, 1] - g["hbar_1_2"]) < tol and abs(Hb[1, 1] - g["hbar_2_2"]) < tol
    assert abs(Hb[2, 1] - g["hbar_3_2"]) < tol
    assert abs(c["cs"][0] - g["alpha_1"]) < tol and abs(c["sn"][0] - g["beta_1"]) < tol
    assert abs(c["cs"][1] - g["alpha_2"]) < tol and abs(c["sn"][1] - g["beta_2"]) < tol
    assert abs(c["s"][0] - g["s_1"]) < tol
    assert abs(c["s"][1] - g["s_2_after_step1"]) < tol
    assert abs(c["arn"][0] - g["arnoldi_res_1"]) < tol and abs(c["arn"][1]) < tol
    R = c["H"]
    assert abs(R[0, 0] - g["r_1_1"]) < tol and abs(R[0, 1] - g["r_1_2"]) < tol
    assert abs(R[1, 1] - g["r_2_2"]) < tol
    assert abs(c["y"][0] - g["y_1"]) < tol and abs(c["y"][1] - g["y_2"]) < tol
    assert abs(c["u"][0] - g["x_1"]) < tol and abs(c["u"][1] - g["x_2"]) < tol


# ---------------------------------------------------------------------------
# Arnoldi process and least-squares problem
# ---------------------------------------------------------------------------

def _cd_small():
    A = I.convdiff2d(8, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 5)
    return A, b


def pin_arnoldi_relation():
    """A V_k = V_{k+1} Hbar_k to 1e-12 (Frobenius, relative to ||A||_F) in
    binary64, for MGS and CGSR."""
    A, b = _cd_small()
    D = _dense(A)
    k = 20
    for ortho in (O.MGS, O.CGSR):
        c = O.arnoldi_cycle(A, b, m=k, ortho=ortho, prec=O.FP64)
        j = c["j"]
        V = c["V"][: j + 1].T
        Hb = c["Hbar"][: j + 1, :j]
        err = np.linalg.norm(D @ V[:, :j] - V @ Hb) / np.linalg.norm(D)
        assert err <= 1e-12, (ortho, err)


def pin_orthonormality():
    """||I - V^T V||_F <= 1e-12 in binary64 for CGSR over the whole cycle and
    <= 1e-4 for a binary32 CGSR basis.  MGS keeps orthogonality only until the
    Arnoldi residual nears working accuracy (Sec. 3): its loss grows like
    u * kappa(A) / (|s_{j+1}| / beta), so the pin checks that product, and the
    1e-12 bound while the relative Arnoldi residual is above 1e-2."""
    A, b = _cd_small()
    beta = np.linalg.norm(b)
    kappa = np.linalg.cond(_dense(A))
    k = 20
    for ortho, prec, tol in ((O.CGSR, O.FP64, 1e-12), (O.CGSR, O.MIXED, 1e-4)):
        c = O.arnoldi_cycle(A, b, m=k, ortho=ortho, prec=prec)
        V = c["V"][: c["j"] + 1]
        err = np.linalg.norm(np.eye(V.shape[0]) - V @ V.T)
        assert err <= tol, (ortho, prec, err)
    c = O.arnoldi_cycle(A, b, m=k, ortho=O.MGS, prec=O.FP64)
    u = 2.0 ** -53
    for j in range(1, c["j"] + 1):
        V = c["V"][: j + 1]
        err = np.linalg.norm(np.eye(j + 1) - V @ V.T)
        rel = c["arn"][j - 1] / beta
        assert err * rel <= 100 * kappa * u, (j, err, rel)
        if rel > 1e-2:
            assert err <= 1e-12, (j, err)


def pin_mgs_equals_cgsr():
    """In exact arithmetic MGS and CGSR give the same Hessenberg matrix; in
    binary64 on a well-conditioned system they agree to 1e-10."""
    A, b = _cd_small()
    c1 = O.arnoldi_cycle(A, b, m=15, ortho=O.MGS, prec=O.FP64)
    c2 = O.arnoldi_cycle(A, b, m=15, ortho=O.CGSR, prec=O.FP64)
    assert c1["j"] == c2["j"]
    d = np.abs(c1["Hbar"] - c2["Hbar"]).max() / np.abs(c1["Hbar"]).max()
    assert d <= 1e-10, d


def pin_arnoldi_step():
    """One inner iteration from a given basis (the replay the full-size GPU
    tests use): in binary64, h_{1..j,j} = V_j^T A v_j (dense numpy), h_{j+1,j}
    = ||A v_j - V_j h||, and v_{j+1} is a unit vector orthogonal to V_j, for
    MGS and CGSR; fed its own cycle's basis, the step reproduces that cycle's
    Hessenberg column and next basis vector in every precision."""
    A, b = _cd_small()
    D = _dense(A)
    for ortho in (O.MGS, O.CGSR):
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64)
        for j in (1, 5, 12):
            V = c["V"][:j]
            h, vn = O.arnoldi_step(A, V, ortho=ortho, prec=O.FP64)
            w = D @ V[-1]
            hx = V @ w
            assert np.allclose(h[:j], hx, rtol=0, atol=1e-13 * np.linalg.norm(w)), (ortho, j)
            assert abs(h[j] - np.linalg.norm(w - V.T @ hx)) <= 1e-12 * np.linalg.norm(w)
            assert abs(np.linalg.norm(vn) - 1.0) <= 1e-13
            assert np.abs(V @ vn).max() <= 1e-12, (ortho, j)
        for prec in (O.MIXED, O.MIXED_FP16, O.MIXED_LIMITED):
            c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=prec)
            for j in (3, 12):
                h, vn = O.arnoldi_step(A, c["V"][:j], ortho=ortho, prec=prec)
                assert np.array_equal(h, c["Hbar"][: j + 1, j - 1]), (ortho, prec, j)
                if j < c["j"]:
                    assert np.array_equal(O.round_basis(vn, prec, len(b)), c["V"][j])


def _f32_exact(a):
    a = np.asarray(a, dtype=np.float64)
    return np.array_equal(a.astype(np.float32).astype(np.float64), a)


def pin_pv_storage():
    """Per-variable precision study (Sec. 4.1): a switch stores exactly its
    variable in binary32.  In one binary64 cycle, the basis switch makes every
    stored basis entry a binary32 value, the Hessenberg switch every entry of
    the unrotated and rotated Hessenberg matrices, the least-squares switch
    the rotations, s and y -- and the other quantities stay genuinely
    binary64.  The A, M and z switches equal the plain binary64 cycle run on
    binary32-rounded A, M and r0 (their definitions), bit for bit; the w
    switch moves the cycle by binary32 roundings only."""
    A, b = _cd_small()
    rp, ci, va = A
    M = (rp, ci, O.spai_values(A, O.spai_jacobi_params()))
    r32 = lambda v: np.asarray(v).astype(np.float32).astype(np.float64)
    for ortho in (O.MGS, O.CGSR):
        base = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64)
        j = base["j"]
        assert not _f32_exact(base["V"][:j]) and not _f32_exact(base["Hbar"][:, :j])
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, pv_mask=O.PV_V)
        assert _f32_exact(c["V"][: j + 1]) and not _f32_exact(c["Hbar"][:, :j])
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, pv_mask=O.PV_H)
        assert _f32_exact(c["Hbar"][:, :j]) and _f32_exact(c["H"][:, :j])
        assert not _f32_exact(c["V"][:j]) and not _f32_exact(c["cs"][:j])
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, pv_mask=O.PV_GIVENS)
        for k in ("cs", "sn", "y"):
            assert _f32_exact(c[k][:j]), k
        assert _f32_exact(c["s"][: j + 1]) and not _f32_exact(c["H"][:, :j])
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, pv_mask=O.PV_A_KRYLOV)
        d = O.arnoldi_cycle((rp, ci, r32(va)), b, m=12, ortho=ortho, prec=O.FP64)
        assert np.array_equal(c["Hbar"], d["Hbar"]) and np.array_equal(c["u"], d["u"])
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, pv_mask=O.PV_Z)
        d = O.arnoldi_cycle(A, r32(b), m=12, ortho=ortho, prec=O.FP64)
        assert np.array_equal(c["Hbar"], d["Hbar"]) and np.array_equal(c["u"], d["u"])
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, M=M, pv_mask=O.PV_M)
        d = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, M=(rp, ci, r32(M[2])))
        assert np.array_equal(c["Hbar"], d["Hbar"]) and np.array_equal(c["u"], d["u"])
        c = O.arnoldi_cycle(A, b, m=12, ortho=ortho, prec=O.FP64, pv_mask=O.PV_W)
        dh = np.abs(c["Hbar"] - base["Hbar"]).max() / np.abs(base["Hbar"]).max()
        assert 0 < dh <= 1e-5, dh


def pin_pv_limited_is_three_switches():
    """The paper's limited mixed solver (Sec. 4.1) is, by its definition, the
    binary64 solver with A for the Krylov step, M and the basis stored in
    binary32: the per-variable switches for those three variables give it bit
    for bit, with and without a preconditioner, for MGS and CGSR."""
    A = I.convdiff2d(20, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 2)
    M = (A[0], A[1], O.spai_values(A, O.spai_jacobi_params()))
    for ortho in (O.MGS, O.CGSR):
        for Mx in (None, M):
            xl, il = O.gmres(A, b, m=20, tol=1e-11, ortho=ortho, prec=O.MIXED_LIMITED,
                             tau=0.0, repeat_first=False, M=Mx, history=True)
            xp, ip = O.gmres(A, b, m=20, tol=1e-11, ortho=ortho, prec=O.FP64, M=Mx,
                             pv_mask=O.PV_A_KRYLOV | O.PV_M | O.PV_V, history=True)
            assert np.array_equal(xl, xp) and np.array_equal(il["arnoldi"], ip["arnoldi"])


def pin_pv_refinement_vs_correction():
    """Sec. 4.1 and Sec. 2: with any one correction variable (A for the Krylov
    step, w, the basis, the Hessenberg matrix, the least-squares vectors, the
    cycle's copy of z) in binary32 the restarted solver still reaches a
    binary64 relative residual of 1e-12; with any one refinement variable (A
    for the residual, b, x, the product A x) in binary32 its true residual
    cannot fall below about the binary32 unit roundoff: it stays above
    u32 / 10 whatever the iteration count."""
    A = I.convdiff2d(30, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 9)
    u32 = 2.0 ** -24
    for ortho in (O.MGS, O.CGSR):
        for bit in (O.PV_A_KRYLOV, O.PV_W, O.PV_V, O.PV_H, O.PV_GIVENS, O.PV_Z):
            _, i = O.gmres(A, b, m=30, tol=1e-12, ortho=ortho, prec=O.FP64, maxiter=2000,
                           pv_mask=bit)
            assert i["converged"] and i["relres"] <= 1e-12, (ortho, bit, i)
        for bit in (O.PV_A_RESID, O.PV_B, O.PV_X, O.PV_AX):
            _, i = O.gmres(A, b, m=30, tol=1e-12, ortho=ortho, prec=O.FP64, maxiter=1500,
                           pv_mask=bit, history=True)
            assert not i["converged"] and min(i["cycle_relres"]) > u32 / 10, (ortho, bit, i)


def pin_givens_least_squares():
    """The rotated problem solves min ||beta e1 - Hbar y|| (checked against
    numpy lstsq), |s_{j+1}| equals that minimum, and it never increases."""
    A, b = _cd_small()
    beta = np.linalg.norm(b)
    for ortho in (O.MGS, O.CGSR):
        c = O.arnoldi_cycle(A, b, m=18, ortho=ortho, prec=O.FP64)
        j = c["j"]
        Hb = c["Hbar"][: j + 1, :j]
        rhs = np.zeros(j + 1)
        rhs[0] = beta
        y, *_ = np.linalg.lstsq(Hb, rhs, rcond=None)
        assert np.allclose(c["y"][:j], y, rtol=1e-11, atol=1e-12 * np.abs(y).max())
        res = np.linalg.norm(rhs - Hb @ y)
        assert abs(c["arn"][j - 1] - res) <= 1e-12 * beta
        arn = c["arn"][:j]
        assert np.all(np.diff(arn) <= 1e-14 * beta)
        # the rotations are orthogonal
        assert np.allclose(c["cs"][:j] ** 2 + c["sn"][:j] ** 2, 1.0, atol=1e-15)


def pin_arnoldi_residual_is_true_residual():
    """Before stagnation, in binary64, |s_{j+1}| = ||r0 - A V_j y_j|| (Saad,
    Prop. 6.9; Sec. 3), checked for every j by brute force."""
    A, b = _cd_small()
    D = _dense(A)
    full = O.arnoldi_cycle(A, b, m=12, ortho=O.CGSR, prec=O.FP64)
    for j in range(1, full["j"] + 1):
        c = O.arnoldi_cycle(A, b, m=12, kmax=j, ortho=O.CGSR, prec=O.FP64)
        true = np.linalg.norm(b - D @ c["u"])
        assert abs(true - full["arn"][j - 1]) <= 1e-10 * max(true, 1e-300) + 1e-14, (j, true)


def pin_tau_restart():
    """Restart strategy 2 (Sec. 3): the cycle ends at the first j with
    |s_{j+1}| <= tau * beta, where the LS residuals come from numpy lstsq."""
    A, b = _cd_small()
    beta = np.linalg.norm(b)
    ref = O.arnoldi_cycle(A, b, m=30, ortho=O.CGSR, prec=O.FP64)
    Hb = ref["Hbar"]
    ls = []
    for j in range(1, ref["j"] + 1):
        rhs = np.zeros(j + 1)
        rhs[0] = beta
        H = Hb[: j + 1, :j]
        y, *_ = np.linalg.lstsq(H, rhs, rcond=None)
        ls.append(np.linalg.norm(rhs - H @ y))
    tau = 1e-3
    expect = next(i + 1 for i, r in enumerate(ls) if r <= tau * beta)
    c = O.arnoldi_cycle(A, b, m=30, ortho=O.CGSR, prec=O.FP64, tau=tau)
    assert c["j"] == expect, (c["j"], expect)


# ---------------------------------------------------------------------------
# precision behaviour (Sec. 2, Sec. 4.1)
# ---------------------------------------------------------------------------

def pin_mixed_reaches_double():
    """With a binary64 residual and update, every mixed form reaches a binary64
    relative residual <= 1e-10 (Sec. 4.1) and the solution matches LAPACK."""
    A = I.convdiff2d(16, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 9)
    xl = np.linalg.solve(_dense(A), b)
    for prec in (O.MIXED, O.MIXED_BF16, O.MIXED_FP16, O.MIXED_LIMITED):
        for ortho in (O.MGS, O.CGSR):
            x, info = O.gmres(A, b, m=30, tol=1e-10, ortho=ortho, prec=prec, maxiter=3000)
            assert info["converged"] and info["relres"] <= 1e-10, (prec, ortho, info)
            assert np.linalg.norm(b - _dense(A) @ x) <= 1e-10 * np.linalg.norm(b)
            assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= 1e-8


def pin_limited_mixed():
    """Sec. 4.1: keeping every operation in binary64 and storing only A (for
    the next Krylov vector) and the basis in binary32 lets MGS improve further
    before it stalls than the fully mixed solver does; the first Arnoldi steps
    agree with binary64 to binary32 accuracy, a basis
    vector it stores is exactly a binary32 number, and the first Hessenberg
    entry is v_1^T A_32 v_1 with A_32 the binary32 rounding of A."""
    A = I.convdiff2d(30, pe=1.0)
    b = I.rhs_ones_noise(A, 1e-3, 1)
    nb = np.linalg.norm(b)
    full = O.arnoldi_cycle(A, b, 100, ortho=O.MGS, prec=O.MIXED)
    lim = O.arnoldi_cycle(A, b, 100, ortho=O.MGS, prec=O.MIXED_LIMITED)
    f64 = O.arnoldi_cycle(A, b, 100, ortho=O.MGS, prec=O.FP64)
    floor_full = full["arn"][: full["j"]].min() / nb
    floor_lim = lim["arn"][: lim["j"]].min() / nb
    assert floor_lim <= 0.1 * floor_full, (floor_lim, floor_full)
    assert floor_lim >= f64["arn"][: f64["j"]].min() / nb
    V = lim["V"][: lim["j"]]
    assert np.array_equal(V, V.astype(np.float32).astype(np.float64))
    rel = np.abs(lim["arn"][:5] - f64["arn"][:5]) / f64["arn"][:5]
    assert rel.max() <= 1e-5
    # the first Hessenberg entry is v_1^T (A_32 v_1) in binary64, A_32 the
    # matrix rounded to binary32 (A itself would differ at ~1e-8)
    A32 = _dense(A).astype(np.float32).astype(np.float64)
    v1 = lim["V"][0]
    h11 = v1 @ (A32 @ v1)
    assert abs(lim["Hbar"][0, 0] - h11) <= 1e-13 * abs(h11)
    assert abs(v1 @ (_dense(A) @ v1) - h11) > 1e-12 * abs(h11)


def _high_np(v):
    """High-order 32 bits of binary64 values by bit masking in numpy."""
    u = np.ascontiguousarray(v, dtype=np.float64).view(np.uint64) & np.uint64(0xFFFFFFFF00000000)
    return u.view(np.float64)


def pin_split_bytes():
    """A stored once as high/low 32-bit halves (Sec. 4 outlook): the high
    part is the value with its low 32 bits cleared (checked against numpy
    bit masking; relative truncation below 2^-20); the Krylov step uses it
    (limited mixed: the first Hessenberg entry is v_1^T A_hi v_1 in binary64);
    binary64 GMRES is unaffected; mixed GMRES on split storage still reaches
    the binary64 target and the LAPACK solution."""
    rng = np.random.default_rng(8)
    v = rng.standard_normal(1000) * np.exp(rng.uniform(-30, 30, 1000))
    hi = np.array([O.high_part(x) for x in v])
    assert np.array_equal(hi, _high_np(v))
    assert np.all(np.abs(v - hi) <= 2.0 ** -20 * np.abs(v))
    A = I.convdiff2d(16, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 9)
    Ahi = _high_np(_dense(A))
    cyc = O.arnoldi_cycle(A, b, 10, ortho=O.MGS, prec=O.MIXED_LIMITED, split_bytes=True)
    v1 = cyc["V"][0]
    h11 = v1 @ (Ahi @ v1)
    assert abs(cyc["Hbar"][0, 0] - h11) <= 1e-13 * abs(h11)
    assert abs(v1 @ (_dense(A).astype(np.float32).astype(np.float64) @ v1) - h11) > 1e-12 * abs(h11)
    c64 = O.arnoldi_cycle(A, b, 10, ortho=O.MGS, prec=O.FP64)
    c64s = O.arnoldi_cycle(A, b, 10, ortho=O.MGS, prec=O.FP64, split_bytes=True)
    assert np.array_equal(c64["Hbar"], c64s["Hbar"])
    xl = np.linalg.solve(_dense(A), b)
    for prec in (O.MIXED, O.MIXED_BF16, O.MIXED_LIMITED):
        x, info = O.gmres(A, b, m=30, tol=1e-10, ortho=O.CGSR, prec=prec, split_bytes=True)
        assert info["converged"] and np.linalg.norm(x - xl) / np.linalg.norm(xl) <= 1e-8


def _lu_dense(LU):
    rp, ci, lu = LU
    n = len(rp) - 1
    L, U = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            (L if ci[k] < i else U)[i, ci[k]] = lu[k]
    return L, U


def pin_ilu0():
    """ILU(0), the paper's preconditioner (Sec. 4): (L U)_ij = a_ij on the
    pattern of A (the defining property of ILU without fill) for a
    convection-diffusion and a random non-symmetric matrix; on a tridiagonal
    matrix (no fill exists) L U = A exactly; the triangular solves equal a
    dense solve with L U."""
    for A in (I.convdiff2d(12, pe=10.0), I.random_dd(40, density=0.15, seed=3)):
        LU = O.ilu0(A)
        L, U = _lu_dense(LU)
        D = _dense(A)
        mask = D != 0
        np.fill_diagonal(mask, True)
        assert np.abs((L @ U - D)[mask]).max() <= 1e-12 * np.abs(D).max()
        assert np.allclose(np.tril(L, -1)[~mask], 0) and np.allclose(U[~mask], 0)
        z = np.random.default_rng(1).standard_normal(len(D))
        assert np.allclose(O.ilu_apply(LU, z), np.linalg.solve(L @ U, z), rtol=1e-12, atol=1e-12)
    n = 30
    rng = np.random.default_rng(2)
    T = np.diag(4 + rng.random(n)) + np.diag(rng.standard_normal(n - 1), 1) + \
        np.diag(rng.standard_normal(n - 1), -1)
    L, U = _lu_dense(O.ilu0(I.dense_to_csr(T)))
    assert np.abs(L @ U - T).max() <= 1e-13


def pin_ilu_left_gmres():
    """Left-preconditioned GMRES (Alg. 1 with M = L U): the first basis
    vector is M^-1 b / ||M^-1 b||; binary64, fully mixed and binary64 with
    the factors in binary32 reach the binary64 residual target on the
    unpreconditioned residual and the LAPACK solution, in fewer inner
    iterations than without the preconditioner."""
    A = I.convdiff2d(20, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 1)
    LU = O.ilu0(A)
    L, U = _lu_dense(LU)
    r = np.linalg.solve(L @ U, b)
    cyc = O.arnoldi_cycle(A, b, 10, ortho=O.MGS, prec=O.FP64, ilu=LU)
    assert np.allclose(cyc["V"][0], r / np.linalg.norm(r), rtol=0, atol=1e-13)
    xl = np.linalg.solve(_dense(A), b)
    _, plain = O.gmres(A, b, m=30, ortho=O.MGS, prec=O.FP64)
    for prec, i32 in ((O.FP64, False), (O.MIXED, False), (O.FP64, True)):
        x, info = O.gmres(A, b, m=30, ortho=O.MGS, prec=prec, ilu=LU, ilu32=i32)
        assert info["converged"] and info["relres"] <= 1e-10
        assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= 1e-8
        assert info["iters"] < plain["iters"] / 2


def pin_negative_control():
    """A residual and update in binary32 cannot pass single-precision accuracy
    (Sec. 2, Sec. 4.1): the all-binary32 solver stalls above 1e-8."""
    A = I.convdiff2d(16, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 9)
    for ortho in (O.MGS, O.CGSR):
        x, info = O.gmres(A, b, m=30, tol=1e-10, ortho=ortho, prec=O.ALL_FP32, maxiter=600)
        assert not info["converged"] and info["relres"] >= 1e-8, info


def pin_monotone_restarts():
    """Each restart cycle minimises the residual over a space that contains the
    zero correction, so the binary64 true residual does not grow from cycle to
    cycle (Sec. 2: ||r_i|| <= delta ||r_{i-1}||)."""
    A = I.convdiff2d(16, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 9)
    for prec in (O.FP64, O.MIXED):
        x, info = O.gmres(A, b, m=8, tol=1e-10, ortho=O.CGSR, prec=prec, maxiter=3000,
                          history=True)
        r = info["cycle_relres"]
        assert len(r) >= 4
        assert np.all(r[1:] <= r[:-1] * (1 + 1e-12)), r


def pin_repeat_first():
    """Restart strategy 1 with the gain-threshold first restart (Sec. 3,
    Sec. 4.2): the first cycle ends on |s_{j+1}| <= tau beta, every later cycle
    runs exactly as long as the first (the last may end early on
    convergence)."""
    A = I.convdiff2d(16, pe=10.0)
    b = I.rhs_ones_noise(A, 1e-3, 9)
    x, info = O.gmres(A, b, m=30, tol=1e-10, ortho=O.CGSR, prec=O.MIXED, maxiter=3000,
                      tau=1e-2, repeat_first=True, history=True)
    k1 = info["first_len"]
    assert k1 < 30
    assert info["iters"] <= k1 * info["restarts"]
    assert info["iters"] > k1 * (info["restarts"] - 1)


# ---------------------------------------------------------------------------
# kernels: SpMV, residual, basis rounding
# ---------------------------------------------------------------------------

def pin_spmv_and_residual():
    """SpMV and residual against dense numpy products: binary64 to 1e-14
    relative; the binary32 SpMV within the sequential-sum bound
    gamma_k u32 sum|a||x| per row, k the row length."""
    A = I.powerlaw_random(300, seed=4)
    D = _dense(A)
    x = np.random.default_rng(1).standard_normal(300)
    y = O.spmv(A, x)
    assert np.allclose(y, D @ x, rtol=1e-14, atol=1e-14 * np.abs(D).sum(1).max())
    y32 = O.spmv(A, x, prec=O.MIXED)
    a32 = D.astype(np.float32).astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    exact = a32 @ x32
    k = np.diff(A[0])
    u = 2.0 ** -24
    bound = (k * u / (1 - k * u)) * (np.abs(a32) @ np.abs(x32))
    assert np.all(np.abs(y32 - exact) <= bound + 1e-300)
    b = np.random.default_rng(2).standard_normal(300)
    z, nrm = O.residual(A, b, x)
    assert np.allclose(z, b - D @ x, rtol=1e-13, atol=1e-13)
    assert abs(nrm - np.linalg.norm(b - D @ x)) <= 1e-13 * nrm


def _bf16_ref(v):
    import torch
    t = torch.tensor(np.asarray(v, np.float32), dtype=torch.float32)
    return t.to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def pin_basis_rounding():
    """bfloat16 storage equals torch's float32 -> bfloat16 conversion
    (round-to-nearest-even, ties included); binary16 storage equals numpy's
    float32 -> float16 conversion of the value scaled by 2^floor(log2(n)/2)."""
    rng = np.random.default_rng(11)
    v = rng.standard_normal(4000) * np.exp(rng.uniform(-20, 5, 4000))
    v = v.astype(np.float32).astype(np.float64)
    # exact ties between bfloat16 neighbours (odd and even kept parts)
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 3.0 + 2.0 ** -7],
                    dtype=np.float64)
    v = np.concatenate([v, ties])
    got = O.round_basis(v, O.MIXED_BF16, 1000)
    assert np.array_equal(got, _bf16_ref(v))
    for n in (1000, 4096, 2_000_000):
        sc = 2.0 ** (int(math.floor(math.log2(n))) // 2)
        w = (rng.standard_normal(3000) / math.sqrt(n)).astype(np.float32)
        w = np.concatenate([w, np.float32([1.0, -1.0, 2.0 ** -30, 5e-8])])
        ref = (w * np.float32(sc)).astype(np.float16).astype(np.float64) / sc
        got = O.round_basis(w.astype(np.float64), O.MIXED_FP16, n)
        assert np.array_equal(got, ref), n
    f32 = O.round_basis(np.array([1.0 + 2.0 ** -30, 0.1]), O.MIXED, 10)
    assert np.array_equal(f32, np.float32([1.0 + 2.0 ** -30, 0.1]).astype(np.float64))


# ---------------------------------------------------------------------------
# learned SpAI preconditioner (loss, gradients, special cases)
# ---------------------------------------------------------------------------

def _spai_case(seed=0, P=3):
    A = I.convdiff3d(3, eps=(0.1, 1.0, 10.0), seed=seed)  # n = 27, anisotropic
    n = len(A[0]) - 1
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((P, n))
    params = rng.standard_normal(O.SPAI_NPARAM) * 0.3
    return A, n, Z, params


def pin_spai_grad_m_fd():
    """dL/dm against central finite differences (L is quadratic in m, so the
    differences are exact up to rounding)."""
    A, n, Z, params = _spai_case(1)
    m = O.spai_values(A, params)
    _, g = O.spai_loss_grad_m(A, m, Z)
    rng = np.random.default_rng(2)
    for k in rng.choice(len(m), 25, replace=False):
        h = 1e-4
        mp = m.copy(); mp[k] += h
        mm = m.copy(); mm[k] -= h
        fd = (O.spai_loss_grad_m(A, mp, Z, grad=False)[0]
              - O.spai_loss_grad_m(A, mm, Z, grad=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])) * 10, (k, fd, g[k])


def pin_spai_grad_params_fd():
    """dL/dparams (chain rule through the MLP and m = g / a_pp) against
    central finite differences, relative 1e-6, on entries of every layer."""
    A, n, Z, params = _spai_case(3)
    _, gp, _ = O.spai_loss_grad(A, params, Z)
    rng = np.random.default_rng(4)
    idx = list(rng.choice(512, 8, replace=False)) + list(512 + rng.choice(64, 4, replace=False))
    idx += list(576 + rng.choice(4096, 10, replace=False)) + list(4672 + rng.choice(64, 4, replace=False))
    idx += list(4736 + rng.choice(64, 6, replace=False)) + [4800]
    for k in idx:
        h = 1e-6 * max(1.0, abs(params[k]))
        pp = params.copy(); pp[k] += h
        pm = params.copy(); pm[k] -= h
        fd = (O.spai_loss_grad(A, pp, Z, grad=False)[0]
              - O.spai_loss_grad(A, pm, Z, grad=False)[0]) / (2 * h)
        assert abs(fd - gp[k]) <= 1e-6 * max(abs(gp[k]), 1e-3 * np.abs(gp).max()), (k, fd, gp[k])


def pin_spai_special_cases():
    """Jacobi parameters give M = D^-1 exactly; zero parameters give M = 0
    and L = ||Z||^2 / (2 P n); the loss scales with the square of the probes."""
    A, n, Z, params = _spai_case(5)
    rp, ci, va = A
    m = O.spai_values(A, O.spai_jacobi_params())
    rows = np.repeat(np.arange(n), np.diff(rp))
    diag = va[rows == ci]
    assert np.array_equal(m[rows == ci], 1.0 / diag)
    assert np.all(m[rows != ci] == 0.0)
    l0, _, _ = O.spai_loss_grad(A, np.zeros(O.SPAI_NPARAM), Z)
    assert abs(l0 - 0.5 * np.sum(Z * Z) / (Z.shape[0] * n)) <= 1e-15 * l0
    l1, _, _ = O.spai_loss_grad(A, params, Z, grad=False)
    l3, _, _ = O.spai_loss_grad(A, params, 3.0 * Z, grad=False)
    assert abs(l3 - 9.0 * l1) <= 1e-12 * l3


def pin_spai_optimum():
    """With the identity as probes, L = ||A M - I||_F^2 / (2 n^2).  The exact
    on-pattern optimum (column-wise least squares, numpy lstsq) is a lower
    bound for every parameter vector, and dL/dm vanishes there."""
    A, n, _, params = _spai_case(6)
    rp, ci, va = A
    D = I.csr_to_dense(A)
    Z = np.eye(n)
    mstar = np.zeros(len(ci))
    rows = np.repeat(np.arange(n), np.diff(rp))
    for q in range(n):
        ks = np.nonzero(ci == q)[0]          # entries of column q of M on A's pattern
        pr = rows[ks]                        # their row indices
        e = np.zeros(n); e[q] = 1.0
        sol, *_ = np.linalg.lstsq(D[:, pr], e, rcond=None)
        mstar[ks] = sol
    lstar, g = O.spai_loss_grad_m(A, mstar, Z)
    fstar = np.sum((D @ I.csr_to_dense((rp, ci, mstar)) - np.eye(n)) ** 2)
    assert abs(lstar - fstar / (2 * n * n)) <= 1e-12 * fstar
    assert np.abs(g).max() <= 1e-12
    for prm in (params, O.spai_jacobi_params(), np.zeros(O.SPAI_NPARAM)):
        l, _, _ = O.spai_loss_grad(A, prm, Z, grad=False)
        assert l >= lstar * (1 - 1e-12)


def pin_spai_feature_invariants():
    """Feature invariants: on the diagonal f0 = f1 = f2 = 1 and f7 = 0; off
    it f2 = 0 and f7 = sign(q - p); f3, f4 >= 1 with the diagonal part of the
    row/column weight; f6 = sign(a)."""
    A = I.powerlaw_random(60, seed=8)
    rp, ci, va = A
    n = len(rp) - 1
    F = O.spai_features(A)
    rows = np.repeat(np.arange(n), np.diff(rp))
    d = rows == ci
    assert np.all(F[d, 0] == 1) and np.all(F[d, 1] == 1) and np.all(F[d, 2] == 1)
    assert np.all(F[d, 7] == 0) and np.all(F[~d, 2] == 0)
    assert np.array_equal(F[~d, 7], np.sign(ci[~d] - rows[~d]))
    assert np.all(F[:, 3] >= 1 - 1e-15) and np.all(F[:, 4] >= 1 - 1e-15)
    assert np.array_equal(F[:, 6], np.sign(va))
    assert np.allclose(F[:, 5], np.diff(rp)[rows] / 8.0)
    # transpose relations: entry (q, p) of A^T sees the column weight of
    # (p, q) as its row weight, the inverse diagonal ratio and the flipped
    # direction
    AT = I.dense_to_csr(I.csr_to_dense(A).T)
    FT = O.spai_features(AT)
    trp, tci, _ = AT
    trows = np.repeat(np.arange(n), np.diff(trp))
    pos = {(int(r), int(c)): k for k, (r, c) in enumerate(zip(trows, tci))}
    for k in range(len(ci)):
        kt = pos[(int(ci[k]), int(rows[k]))]
        assert abs(FT[kt, 3] - F[k, 4]) <= 1e-14 * F[k, 4]
        assert abs(FT[kt, 1] * F[k, 1] - 1.0) <= 1e-14
        assert FT[kt, 7] == -F[k, 7]


def pin_adam_first_step():
    """The first Adam step moves every parameter with a nonzero gradient by
    lr * sign(g) (m/(1-b1) = g and sqrt(v/(1-b2)) = |g|, up to eps), and leaves
    a zero-gradient parameter unchanged."""
    p = np.array([1.0, 1.0, 1.0, -2.0])
    g = np.array([1.0, -2.0, 0.0, 3e-3])
    p1, m1, v1 = O.adam_step(p, np.zeros(4), np.zeros(4), g, 1, 0.1)
    assert np.allclose(p1, [0.9, 1.1, 1.0, -2.1], rtol=0, atol=1e-6)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def _cyclic(n):
    P = np.zeros((n, n))
    for i in range(n):
        P[(i + 1) % n, i] = 1.0
    b = np.zeros(n)
    b[0] = 1.0
    return I.dense_to_csr(P), b


def pin_stall_restart():
    """Third strategy (Sec. 3): on the cyclic shift the Arnoldi residual stays
    exactly 1 for n-1 steps (complete stagnation), so with a window of w
    iterations the first possible test, at iteration w, already sees no gain
    and ends the cycle there; a factor of 1 (no gain needed) never triggers,
    and neither does the default off."""
    A, b = _cyclic(16)
    for w in (1, 3, 5):
        for ortho in (O.MGS, O.CGSR):
            cyc = O.arnoldi_cycle(A, b, m=16, ortho=ortho, prec=O.FP64, stall_factor=1.001,
                                  stall_window=w)
            assert cyc["j"] == w, (w, cyc["j"])
    assert O.arnoldi_cycle(A, b, m=16, prec=O.FP64, stall_factor=1.0, stall_window=2)["j"] == 16
    assert O.arnoldi_cycle(A, b, m=16, prec=O.FP64)["j"] == 16
    # default window: ceil(0.05 m)
    x, info = O.gmres(A, b, m=40, prec=O.FP64, stall_factor=1.001, maxiter=10)
    assert info["first_len"] == 2 and info["iters"] == 10
    # a real stall (mixed MGS, binary32 basis): the cycle ends at the first
    # iteration whose residual is within the factor of the one w steps back
    # in the history of the same cycle run without the test
    A2 = I.convdiff2d(30, pe=1.0)
    b2 = I.rhs_ones_noise(A2, 1e-3, 1)
    full = O.arnoldi_cycle(A2, b2, m=100, ortho=O.MGS, prec=O.MIXED)
    hist = np.concatenate([[np.linalg.norm(b2)], full["arn"][: full["j"]]])
    for w in (3, 5, 8):
        want = next(j for j in range(w, 101) if hist[j - w] < 1.001 * hist[j])
        cyc = O.arnoldi_cycle(A2, b2, m=100, ortho=O.MGS, prec=O.MIXED, stall_factor=1.001,
                              stall_window=w)
        assert cyc["j"] == want < 100, (w, cyc["j"], want)


def pin_s_matrix():
    """Fourth strategy (Sec. 3): ||S_k|| of S_k = (I + U_k)^-1 U_k, U_k the
    strictly upper part of V_k^T V_k.  The Frobenius norms the cycle reports
    equal those of S formed densely (numpy solve) from the basis it exports;
    the spectral estimate is the power method's, bounded by the exact 2-norm
    and converging to it with more iterations; an orthonormal binary64 CGSR
    basis has ||S|| ~ 0; unit vectors with a repeated one give ||S||_2 = 1
    (Paige: S is a contraction for unit columns, of norm 1 exactly when they
    are dependent)."""
    A = I.convdiff2d(12, pe=5.0)
    b = I.rhs_ones_noise(A, 1e-3, 2)
    cyc = O.arnoldi_cycle(A, b, m=30, ortho=O.MGS, prec=O.MIXED, orth_norm=O.ORTH_FROBENIUS,
                          orth_threshold=10.0)
    j = cyc["j"]
    assert j >= 10
    for c in (1, 4, j - 1):
        k = c + 2
        Vk = cyc["V"][:k].T
        U = np.triu(Vk.T @ Vk, 1)
        S = np.linalg.solve(np.eye(k) + U, U)
        assert abs(cyc["orth"][c] - np.linalg.norm(S, "fro")) <= 1e-9 * max(1e-300, cyc["orth"][c]) + 1e-15
    rng = np.random.default_rng(4)
    for k in (3, 7, 20):
        S = np.triu(rng.standard_normal((k, k)), 1)
        exact = np.linalg.norm(S, 2)
        assert O.s_norm2(S, 10) <= exact * (1 + 1e-12)
        assert abs(O.s_norm2(S, 2000) - exact) <= 1e-8 * exact
    # orthonormal basis: S ~ 0
    cyc = O.arnoldi_cycle(A, b, m=30, ortho=O.CGSR, prec=O.FP64, orth_norm=O.ORTH_SPECTRAL,
                          orth_threshold=10.0)
    assert np.max(cyc["orth"][: cyc["j"]]) <= 1e-12
    # dependent unit vectors: ||S||_2 = 1
    v = rng.standard_normal((5, 40))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v[4] = v[1]
    U = np.triu(v @ v.T, 1)
    S = np.linalg.solve(np.eye(5) + U, U)
    assert abs(O.s_norm2(S, 3000) - 1.0) <= 1e-6


def pin_orthogonality_loss_restart():
    """Mixed MGS on a fast-converging system: the binary32 basis loses
    independence as the Arnoldi residual stalls, ||S_k||_2 climbs to 1
    (Sec. 4.1 observes the same), and a threshold ends the cycle at the first
    iteration whose norm reaches it."""
    A = I.convdiff2d(30, pe=1.0)
    b = I.rhs_ones_noise(A, 1e-3, 1)
    full = O.arnoldi_cycle(A, b, m=100, ortho=O.MGS, prec=O.MIXED, orth_norm=O.ORTH_SPECTRAL,
                           orth_threshold=10.0)
    orth, arn = full["orth"][: full["j"]], full["arn"][: full["j"]]
    assert full["j"] == 100 and orth[-1] >= 0.99 and orth[-1] <= 1 + 1e-5
    assert arn[-1] >= 0.999 * arn[-10]  # stalled
    assert orth[5] <= 1e-3
    for thr in (0.1, 0.5, 0.9):
        first = int(np.argmax(orth >= thr))
        cyc = O.arnoldi_cycle(A, b, m=100, ortho=O.MGS, prec=O.MIXED,
                              orth_norm=O.ORTH_SPECTRAL, orth_threshold=thr)
        assert cyc["j"] == first + 1, (thr, cyc["j"], first)


ALL_PINS = [
    pin_lu_fp64, pin_exact_convergence, pin_identity, pin_diag_distinct, pin_cyclic_shift,
    pin_hand_2x2, pin_arnoldi_relation, pin_orthonormality, pin_mgs_equals_cgsr,
    pin_givens_least_squares, pin_arnoldi_residual_is_true_residual, pin_tau_restart,
    pin_mixed_reaches_double, pin_negative_control, pin_monotone_restarts, pin_repeat_first,
    pin_spmv_and_residual, pin_basis_rounding,
    pin_spai_grad_m_fd, pin_spai_grad_params_fd, pin_spai_special_cases, pin_spai_optimum,
    pin_spai_feature_invariants, pin_adam_first_step, pin_stall_restart, pin_s_matrix,
    pin_orthogonality_loss_restart, pin_limited_mixed, pin_split_bytes, pin_ilu0,
    pin_ilu_left_gmres, pin_arnoldi_step, pin_pv_storage, pin_pv_limited_is_three_switches,
    pin_pv_refinement_vs_correction,
]

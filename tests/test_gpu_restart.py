"""Restart strategies three and four of Sec. 3 on the GPU (marker: gpu).

Third: end the cycle once the Arnoldi residual improved by less than a
factor over the last w inner iterations.  Fourth: end it once the norm of
S_k = (I + U_k)^-1 U_k (U_k the strictly upper part of V_k^T V_k) reaches a
threshold.  Checked against the oracle's cycle and against the textbook
special case (complete stagnation on the cyclic shift), and the monitor's
norms against S formed densely from the basis the GPU exports.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=torch.float64)


def _cyclic(n):
    P = np.zeros((n, n))
    for i in range(n):
        P[(i + 1) % n, i] = 1.0
    b = np.zeros(n)
    b[0] = 1.0
    return I.dense_to_csr(P), b


@pytest.mark.parametrize("path", ["grid", "block"])
@pytest.mark.parametrize("w", [1, 3, 5])
def test_stall_on_cyclic_shift(path, w, gpulib):
    """Complete stagnation: the first possible test, at iteration w, sees no
    gain, so every cycle has length w (as in the oracle)."""
    A, b = _cyclic(16)
    s = G.Solver(A)
    s.set_opts(path=G.PATH_GRID if path == "grid" else G.PATH_BLOCK, stall_factor=1.001,
               stall_window=w)
    x, st, info = s.solve(b, np.zeros(16), m=16, ortho="mgs", prec="fp64", maxiter=4 * w)
    s.close()
    xo, io = O.gmres(A, b, m=16, ortho=O.MGS, prec=O.FP64, stall_factor=1.001, stall_window=w,
                     maxiter=4 * w)
    assert info["first_len"] == io["first_len"] == w
    assert info["iters"] == io["iters"] == 4 * w and info["restarts"] == 4


def _stall_case():
    A = I.convdiff2d(30, pe=1.0)
    return A, I.rhs_ones_noise(A, 1e-3, 1)


@pytest.mark.parametrize("ortho", ["mgs", "cgsr"])
def test_stall_cycle_follows_its_history(ortho, gpulib):
    """Mixed precision, a real stall: the GPU cycle ends at the first
    iteration where its own Arnoldi residual history meets the stall rule.
    Against the oracle the stall point agrees to 25 %: where a binary32
    basis stalls depends on the rounding of its inner products, which the
    GPU sums by trees (error ~ log2(n) u) and the oracle sequentially
    (~ n u), so the GPU basis stays independent a little longer."""
    A, b = _stall_case()
    n = len(b)
    s = G.Solver(A)
    full = G.gmres_arnoldi(s.h, dev(b), 100, 100, G.ORTHOS[ortho], G.MIXED, n=n)
    s.set_opts(stall_factor=1.001, stall_window=5)
    cyc = G.gmres_arnoldi(s.h, dev(b), 100, 100, G.ORTHOS[ortho], G.MIXED, n=n)
    s.close()
    hist = np.concatenate([[np.linalg.norm(b)], full["arn"][: full["j"]]])
    want = next((j for j in range(5, full["j"] + 1) if hist[j - 5] < 1.001 * hist[j]), 100)
    assert cyc["j"] == want, (cyc["j"], want)
    oc = O.arnoldi_cycle(A, b, 100, ortho=O.MGS if ortho == "mgs" else O.CGSR, prec=O.MIXED,
                         stall_factor=1.001, stall_window=5)
    assert abs(cyc["j"] - oc["j"]) <= 0.25 * oc["j"], (cyc["j"], oc["j"])
    if ortho == "mgs":
        assert cyc["j"] < 100  # mixed MGS stalls inside a 100-step cycle


@pytest.mark.parametrize("norm", ["frobenius", "spectral"])
@pytest.mark.parametrize("prec", ["mixed", "mixed_fp16"])
def test_orth_monitor_norms(norm, prec, gpulib):
    """The monitor's ||S_k|| equal those of S formed densely (numpy) from the
    basis the GPU stored, to the accuracy of the binary32 inner products; the
    spectral estimate never exceeds the exact 2-norm by more than that."""
    A, b = _stall_case()
    n = len(b)
    kind = G.ORTH_FROBENIUS if norm == "frobenius" else G.ORTH_SPECTRAL
    s = G.Solver(A)
    s.set_opts(orth_norm=kind, orth_threshold=10.0)
    cyc = G.gmres_arnoldi(s.h, dev(b), 100, 100, G.ORTHO_MGS, G.PRECISIONS[prec], n=n)
    got = G.gmres_orth_norms(s.h, 100)
    s.close()
    j = cyc["j"]
    assert j == 100
    V = cyc["V"]
    for c in (0, 10, 40, 70, 98):
        k = c + 2
        Vk = V[:k].T
        U = np.triu(Vk.T @ Vk, 1)
        S = np.linalg.solve(np.eye(k) + U, U)
        if kind == G.ORTH_FROBENIUS:
            ref = np.linalg.norm(S, "fro")
            assert abs(got[c] - ref) <= 2e-3 * ref + 5e-5, (c, got[c], ref)
        else:
            ref = O.s_norm2(S, 10)
            assert abs(got[c] - ref) <= 2e-3 * ref + 5e-5, (c, got[c], ref)
            assert got[c] <= np.linalg.norm(S, 2) * (1 + 2e-3) + 5e-5
    # the binary32 basis loses independence as the cycle stalls (Sec. 4.1)
    assert got[98] >= 0.9


def test_orth_restart_and_solve(gpulib):
    """A threshold ends the cycle at the first iteration whose norm reaches
    it (from the GPU's own history); the restarted solve with the test on
    converges to the binary64 target; the oracle's first cycle ends within
    25 % of the GPU's (the binary32 basis loses independence at a point set
    by the rounding of its inner products: tree sums on the GPU, sequential
    ones in the oracle)."""
    A, b = _stall_case()
    n = len(b)
    s = G.Solver(A)
    s.set_opts(orth_norm=G.ORTH_SPECTRAL, orth_threshold=10.0)
    G.gmres_arnoldi(s.h, dev(b), 100, 100, G.ORTHO_MGS, G.MIXED, n=n)
    hist = G.gmres_orth_norms(s.h, 100)
    s.set_opts(orth_threshold=0.5)
    cyc = G.gmres_arnoldi(s.h, dev(b), 100, 100, G.ORTHO_MGS, G.MIXED, n=n)
    first = int(np.argmax(hist >= 0.5))
    assert hist[first] >= 0.5 and cyc["j"] == first + 1
    oc = O.arnoldi_cycle(A, b, 100, ortho=O.MGS, prec=O.MIXED, orth_norm=O.ORTH_SPECTRAL,
                         orth_threshold=0.5)
    assert abs(cyc["j"] - oc["j"]) <= 0.25 * oc["j"], (cyc["j"], oc["j"])
    s.set_opts(repeat_first=0, tau=0.0)
    x, st, info = s.solve(b, np.zeros(n), m=100, ortho="mgs", prec="mixed", maxiter=5000)
    assert st == G.OK and info["path"] == G.PATH_GRID
    assert O.residual_norm(A, b, x) / np.linalg.norm(b) <= 1e-10
    assert info["first_len"] == cyc["j"]
    s.close()


def test_orth_options_checked(gpulib):
    A, b = _stall_case()
    s = G.Solver(A)
    s.set_opts(path=G.PATH_BLOCK, orth_norm=G.ORTH_SPECTRAL)
    with pytest.raises(G.GmresError) as e:
        s.solve(b, np.zeros(len(b)), m=30, ortho="mgs", prec="mixed")
    assert e.value.status == G.ERR_ARG
    o = G.gmres_get_opts(s.h)
    o.path, o.orth_norm, o.orth_threshold = G.PATH_AUTO, G.ORTH_SPECTRAL, 0.0
    with pytest.raises(G.GmresError):
        G.gmres_set_opts(s.h, o)
    s.close()

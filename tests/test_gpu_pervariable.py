"""Per-variable precision switches on the GPU (marker: gpu).

Sec. 4.1 stores one solver variable at a time in binary32 while the rest of
the binary64 solver is unchanged (gmres_opts.pv_mask).  Checked against the
oracle's implementation of the same switches:

* one restart cycle per switch (MGS and CGSR) element by element, and the
  switched variable is really stored in binary32 on the GPU (every exported
  value of it is a binary32 value, the unswitched ones are not);
* whole solves: with any correction variable in binary32 the solver reaches a
  binary64 relative residual of 1e-12 like the oracle; with any refinement
  variable (A for the residual, b, x, A x) in binary32 the true residual
  stalls above 1e-8 on the GPU as in the oracle -- the paper's prediction
  that a residual or an update in single precision cannot pass single
  accuracy (Sec. 2), shown on the GPU.
"""
import numpy as np
import pytest

import oracle as O
from paper_2011_01850_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2011_01850_gb300 import gmres as G

CORRECTION = [("a_krylov", O.PV_A_KRYLOV), ("v", O.PV_V), ("w", O.PV_W), ("h", O.PV_H),
              ("givens", O.PV_GIVENS), ("z", O.PV_Z)]
REFINEMENT = [("a_resid", O.PV_A_RESID), ("b", O.PV_B), ("x", O.PV_X), ("ax", O.PV_AX)]
# A one-ulp difference of a binary32 rounding (the two sides sum in different
# orders, so a binary64 value can land on either side of a binary32 rounding
# boundary) is 2^-24 relative; over 12 inner iterations such differences stay
# within the binary32 cycle tolerance of the other parity tests.
CYCLE_TOL = 2e-4


def _f32_exact(a):
    a = np.asarray(a, dtype=np.float64)
    return np.array_equal(a.astype(np.float32).astype(np.float64), a)


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name,bit", CORRECTION, ids=[c[0] for c in CORRECTION])
@pytest.mark.parametrize("ortho", [O.MGS, O.CGSR], ids=["mgs", "cgsr"])
def test_pervariable_cycle_parity(name, bit, ortho, gpulib):
    A = I.convdiff2d(33, 31, pe=10.0)  # n = 1023: several blocks and a ragged tail
    b = I.rhs_ones_noise(A, 1e-3, 4)
    n = len(b)
    m, kmax = 24, 12
    s = G.Solver(A, stream=torch.cuda.current_stream())
    s.set_opts(pv_mask=bit)
    g = G.gmres_arnoldi(s.h, _dev(b), m, kmax, ortho, G.FP64, n=n)
    s.close()
    o = O.arnoldi_cycle(A, b, m, ortho=ortho, prec=O.FP64, kmax=kmax, pv_mask=bit)
    assert g["j"] == o["j"] == kmax
    j = kmax
    beta = np.linalg.norm(b)

    def close(a, b_, scale, what):
        err = np.abs(a - b_).max() / scale
        assert err <= CYCLE_TOL, (name, what, err)

    close(g["Hbar"][: j + 1, :j], o["Hbar"][: j + 1, :j], np.abs(o["Hbar"]).max(), "Hbar")
    close(g["H"][: j + 1, :j], o["H"][: j + 1, :j], np.abs(o["H"]).max(), "H")
    close(g["cs"][:j], o["cs"][:j], 1.0, "cs")
    close(g["sn"][:j], o["sn"][:j], 1.0, "sn")
    close(g["s"][: j + 1], o["s"][: j + 1], beta, "s")
    close(g["y"][:j], o["y"][:j], np.abs(o["y"][:j]).max(), "y")
    close(g["u"], o["u"], np.abs(o["u"]).max(), "u")
    close(g["V"][:j], o["V"][:j], np.abs(o["V"][:j]).max(), "V")
    # the switch stores its variable, and only it, in binary32 on the GPU
    stored = {O.PV_V: [g["V"][: j + 1]], O.PV_H: [g["Hbar"][:, :j], g["H"][:, :j]],
              O.PV_GIVENS: [g["cs"][:j], g["sn"][:j], g["s"][: j + 1], g["y"][:j]]}
    for vb, arrays in stored.items():
        for a in arrays:
            assert _f32_exact(a) == (vb == bit), (name, vb)


@pytest.fixture(scope="module")
def system():
    A = I.convdiff3d(14, seed=2)      # n = 2744
    b = I.rhs_ones_noise(A, 1e-3, 11)
    return A, b


def _resid_bound(A, b, x):
    rp, ci, va = A
    n = len(b)
    k = int(np.diff(rp).max()) + 1
    ax = np.zeros(n)
    np.add.at(ax, np.repeat(np.arange(n), np.diff(rp)), np.abs(va) * np.abs(x[ci]))
    u = 2.0 ** -53
    return 2 * k * u / (1 - k * u) * np.linalg.norm(ax + np.abs(b)) / np.linalg.norm(b)


def _solve(A, b, mask, ortho, maxiter, precond=None):
    n = len(b)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    if precond is not None:
        G.gmres_spai_set(s.h, precond)
        s.set_opts(precond=G.PRECOND_SPAI, fallback=0)
    s.set_opts(pv_mask=mask)
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, st, info = s.solve(_dev(b), dx, m=30, tol=1e-12, ortho=ortho, prec="fp64",
                          maxiter=maxiter)
    s.close()
    return dx.cpu().numpy(), st, info


@pytest.mark.parametrize("name,bit", CORRECTION + [("m", O.PV_M)],
                         ids=[c[0] for c in CORRECTION] + ["m"])
@pytest.mark.parametrize("ortho", ["mgs", "cgsr"])
def test_pervariable_correction_reaches_double(system, name, bit, ortho, gpulib):
    A, b = system
    pre = np.asarray(O.spai_jacobi_params(), np.float32) if bit == O.PV_M else None
    x, st, info = _solve(A, b, bit, ortho, 2000, precond=pre)
    assert st == G.OK, (name, info)
    rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
    assert rel <= 1e-12, (name, rel)
    # two binary64 evaluations of z = b - A x differ by at most
    # 2 gamma_{k+1} (|A||x| + |b|) per entry (k entries per row)
    assert abs(rel - info["relres"]) <= _resid_bound(A, b, x), (rel, info["relres"])
    M = (A[0], A[1], O.spai_values(A, O.spai_jacobi_params())) if pre is not None else None
    xo, oi = O.gmres(A, b, m=30, tol=1e-12, ortho=O.MGS if ortho == "mgs" else O.CGSR,
                     prec=O.FP64, maxiter=2000, pv_mask=bit, M=M)
    assert oi["converged"]
    assert abs(info["iters"] - oi["iters"]) <= 30, (info["iters"], oi["iters"])
    # kappa_2 of this 14^3 system is about 0.4 * 15^2 = 90: both x within
    # kappa (rel + rel_o) of each other
    err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
    assert err <= 200 * (rel + oi["relres"]), err


@pytest.mark.parametrize("name,bit", REFINEMENT + [("all", O.PV_CORRECTION | O.PV_REFINEMENT)],
                         ids=[c[0] for c in REFINEMENT] + ["all"])
def test_pervariable_refinement_stalls(system, name, bit, gpulib):
    """The GPU negative control: a refinement variable in binary32 keeps the
    true binary64 residual above 1e-8, as in the oracle, for as many inner
    iterations as it is given."""
    A, b = system
    x, st, info = _solve(A, b, bit & ~O.PV_M, "cgsr", 1500)
    assert st == G.MAXITER, (name, st, info)
    assert not info["converged"]
    rel = O.residual_norm(A, b, x) / np.linalg.norm(b)
    assert abs(rel - info["relres"]) <= _resid_bound(A, b, x)
    assert rel > 1e-8, (name, rel)
    _, oi = O.gmres(A, b, m=30, tol=1e-12, ortho=O.CGSR, prec=O.FP64, maxiter=1500,
                    pv_mask=bit & ~O.PV_M)
    assert not oi["converged"]
    assert oi["relres"] / 3 <= rel <= 3 * oi["relres"], (name, rel, oi["relres"])


def test_pervariable_arguments(system, gpulib):
    A, b = system
    n = len(b)
    s = G.Solver(A, stream=torch.cuda.current_stream())
    s.set_opts(pv_mask=O.PV_V)
    dx = torch.zeros(n, dtype=torch.float64, device="cuda")
    for prec in ("mixed", "mixed_limited"):
        with pytest.raises(G.GmresError) as e:
            s.solve(_dev(b), dx, m=30, tol=1e-10, ortho="cgsr", prec=prec, maxiter=10)
        assert e.value.status == G.ERR_ARG
    s.set_opts(path=G.PATH_BLOCK)
    with pytest.raises(G.GmresError) as e:
        s.solve(_dev(b), dx, m=30, tol=1e-10, ortho="cgsr", prec="fp64", maxiter=10)
    assert e.value.status == G.ERR_ARG
    with pytest.raises(G.GmresError):
        s.set_opts(pv_mask=4096)
    s.close()

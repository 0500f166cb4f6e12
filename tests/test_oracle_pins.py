"""The CPU oracle against its pins, and planted mistakes against the pins.

Runs on any CPU host (marker: not gpu).  The planted-mistake tests copy the
oracle sources to a temporary directory, apply one textual mistake of the kind
a restatement of Algorithm 1 could plausibly contain (a flipped sign, a wrong
index, a dropped term, a transposed operand), compile that copy with gcc and
check that at least one pin rejects it.
"""
from __future__ import annotations

import os
import shutil
import warnings

import pytest

import oracle as O
import oracle_pins as P

ORACLE_DIR = os.path.dirname(os.path.abspath(O.__file__))


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


# (file, exact text, replacement, what the mistake is)
MUTATIONS = [
    ("cycle_impl.inc", "s[c + 1] = -be * sj;", "s[c + 1] = be * sj;",
     "sign of the new s_{j+1}"),
    ("cycle_impl.inc", "col[i + 1] = -sn[i] * hi + cs[i] * hi1;",
     "col[i + 1] = sn[i] * hi + cs[i] * hi1;", "sign in applying an old rotation"),
    ("cycle_impl.inc", "col[i] = cs[i] * hi + sn[i] * hi1;",
     "col[i] = cs[i] * hi + sn[i + 1] * hi1;", "wrong rotation index"),
    ("cycle_impl.inc", "be = hj1 / rho;", "be = hjj / rho;", "rotation formed from wrong entry"),
    ("cycle_impl.inc", "s[c] = al * sj;", "s[c] = sj;", "dropped rotation of s_j"),
    ("cycle_impl.inc", "acc -= H[(size_t)l * ld + i] * y[l];",
     "acc -= H[(size_t)i * ld + l] * y[l];", "transposed triangle in back substitution"),
    ("cycle_impl.inc", "for (int32_t l = i + 1; l < j; ++l)",
     "for (int32_t l = i + 2; l < j; ++l)", "dropped term in back substitution"),
    ("cycle_impl.inc", "V[(size_t)(c + 1) * n + r] = (R)orc_store(w[r] / hnext, vprec, n);",
     "V[(size_t)(c + 1) * n + r] = (R)orc_store(w[r], vprec, n);", "v_{j+1} not normalised"),
    ("cycle_impl.inc", "V[r] = (R)orc_store(rr[r] / beta, vprec, n);",
     "V[r] = (R)orc_store(rr[r], vprec, n);", "v_1 not normalised"),
    ("cycle_impl.inc", "for (int32_t i = 0; i < j; ++i) {\n        const R *v = V + (size_t)i * n;",
     "for (int32_t i = 0; i + 1 < j; ++i) {\n        const R *v = V + (size_t)i * n;",
     "MGS skips the last projection"),
    ("cycle_impl.inc", "FN(cgs_pass)(n, j, V, w, g2, pv);\n", "",
     "CGSR without its second pass"),
    ("cycle_impl.inc", "Hb[(size_t)c * ld + c + 1] = hnext;", "Hb[(size_t)c * ld + c + 1] = wnorm0;",
     "subdiagonal from the wrong norm"),
    ("cycle_impl.inc", "acc += a[k] * x[colind[k]];\n        y[i] = acc;",
     "acc += a[k] * x[i];\n        y[i] = acc;", "SpMV gathers the wrong operand"),
    ("gmres_oracle.c", "double zi = b[i] - acc;", "double zi = b[i] + acc;",
     "residual sign"),
    ("gmres_oracle.c", "x[i] = x[i] + u[i];", "x[i] = x[i] - u[i];", "update sign"),
    ("gmres_oracle.c", "bits += 0x7fffu + lsb;", "bits += 0x8000u;",
     "bfloat16 ties away from even"),
    ("gmres_oracle.c", "return ldexp(1.0, lg / 2);", "return ldexp(1.0, lg);",
     "binary16 scale"),
    ("gmres_oracle.c", "return (double)(float)v;\n", "return v;\n",
     "binary32 basis not rounded"),
    ("cycle_impl.inc", "acc -= U[(size_t)l * ld + i] * scol[l];", "",
     "S taken as U (inverse of I + U dropped)"),
    ("cycle_impl.inc", "ah[j - rs->stall_window] < rs->stall_factor * arnres",
     "ah[j - rs->stall_window + 1] < rs->stall_factor * arnres", "stall window one short"),
    ("cycle_impl.inc", "ah[j - rs->stall_window] < rs->stall_factor * arnres",
     "ah[j - rs->stall_window] < arnres", "stall factor dropped"),
    ("gmres_oracle.c", "acc += S[(size_t)l * ld + i] * yv[i];",
     "acc += S[(size_t)i * ld + l] * yv[i];", "power method multiplies by S, not S^T"),
    ("gmres_oracle.c", "a[k] = !limited ? pv32(", "a[k] = 1 ? pv32(",
     "limited mode keeps A in binary64"),
    ("gmres_oracle.c", "u &= 0xFFFFFFFF00000000ull;", "u &= 0xFFFFFFFFF0000000ull;",
     "high part keeps four low-order bits"),
    ("gmres_oracle.c", "(rs->split_bytes ? orc_high_part(vals[k]) : (double)(float)vals[k])",
     "(double)(float)vals[k]", "split storage ignored in the Krylov step"),
    ("ilu_oracle.c", "lu[p] = lu[p] / pivot; /* l_ik */", "lu[p] = lu[p]; /* l_ik */",
     "ILU(0) without the division by the pivot"),
    ("ilu_oracle.c", "lu[q] = lu[q] - lu[p] * lu[kj];", "lu[q] = lu[q] + lu[p] * lu[kj];",
     "ILU(0) update sign"),
    ("cycle_impl.inc", "FN(ilu_apply)(n, pm_rowptr, pm_colind, pm, rr, rl);\n        rr = rl;",
     "", "left preconditioner not applied to the residual"),
    ("cycle_impl.inc", "for (int32_t p = rowptr[i]; p < rowptr[i + 1] && colind[p] < i; ++p)\n            acc -= lu[p] * out[colind[p]];",
     "for (int32_t p = rowptr[i]; p < rowptr[i + 1] && colind[p] <= i; ++p)\n            acc -= lu[p] * out[colind[p]];",
     "forward substitution takes in the diagonal"),
    ("cycle_impl.inc", "FN(spmv)(n, rowptr, colind, a, V + (size_t)(ncols - 1) * n, w);",
     "FN(spmv)(n, rowptr, colind, a, V, w);", "replayed step multiplies v_1, not v_j"),
    ("gmres_oracle.c", "x[i] = x[i] + u[i];\n                x[i] = pv32(x[i], pvr, ORC_PV_X);",
     "x[i] = x[i] + u[i];", "solution switch not applied to the update"),
    ("cycle_impl.inc", "hij = PV(hij, ORC_PV_H);", "hij = PV(hij, ORC_PV_W);",
     "MGS coefficient rounded under the w switch"),
    ("cycle_impl.inc", "const int32_t vprec = (pv & ORC_PV_V) ? ORC_MIXED : prec;",
     "const int32_t vprec = prec;", "basis switch ignored"),
    ("gmres_oracle.c", "ar[k] = pv32(vals[k], pvr, ORC_PV_A_RESID);", "ar[k] = vals[k];",
     "residual keeps binary64 A under its switch"),
    ("spai_oracle.c", "atr[colind[k]] += vals[k] * r[i];", "atr[i] += vals[k] * r[colind[k]];",
     "A instead of A^T in the preconditioner gradient"),
    ("spai_oracle.c", "d2[o] = z2[o] > 0 ? dgk * params[P_W3 + o] : 0;",
     "d2[o] = dgk * params[P_W3 + o];", "missing ReLU derivative"),
    ("spai_oracle.c", "const double dgk = gm[k] / dg[p];", "const double dgk = gm[k];",
     "chain rule through m = g / a_pp dropped"),
    ("spai_oracle.c", "f[4] = cs[q] / fabs(d[q]);", "f[4] = rs[q] / fabs(d[q]);",
     "row weight used as column weight"),
]


@pytest.mark.parametrize("mut", MUTATIONS, ids=[m[3] for m in MUTATIONS])
def test_planted_mistake_is_caught(mut, tmp_path):
    fname, old, new, what = mut
    src = tmp_path / "src"
    src.mkdir()
    for f in os.listdir(ORACLE_DIR):
        if f.endswith((".c", ".h", ".inc")):
            shutil.copy(os.path.join(ORACLE_DIR, f), src / f)
    text = (src / fname).read_text()
    assert text.count(old) >= 1, "mutation anchor missing: " + what
    (src / fname).write_text(text.replace(old, new, 1))
    so = O.build(force=True, src_dir=str(src), out_path=str(tmp_path / "mutant.so"))
    L = O.load_path(so)
    caught = []
    with O.use(L), warnings.catch_warnings():
        warnings.simplefilter("ignore")
        for pin in P.ALL_PINS:
            try:
                pin()
            except Exception:  # any failure of the pin rejects the mutant
                caught.append(pin.__name__)
    assert caught, "planted mistake not caught by any pin: " + what

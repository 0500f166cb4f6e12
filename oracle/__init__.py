"""CPU oracle for restarted mixed-precision GMRES(m) -- test infrastructure only.

This package wraps ``gmres_oracle.c`` (a plain, single-threaded restatement of
Algorithm 1 of Lindquist, Luszczek and Dongarra, arXiv 2011.01850) through
ctypes.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the CUDA library never does, and the two
share no code.

The shared object is compiled with gcc on first use (or by ``build()``) into
``oracle/liboracle.so``; it is rebuilt whenever a source file is newer.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["gmres_oracle.c", "gmres_oracle.h", "cycle_impl.inc", "spai_oracle.c", "ilu_oracle.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MGS, CGSR = 0, 1
ORTH_OFF, ORTH_SPECTRAL, ORTH_FROBENIUS = 0, 1, 2
FP64, MIXED, MIXED_BF16, MIXED_FP16, ALL_FP32, MIXED_LIMITED = 0, 1, 2, 3, 4, 5
# per-variable precision switches (gmres_oracle.h, Sec. 4.1): bit set = that
# variable stored in binary32, the rest of the binary64 solver unchanged
PV_A_KRYLOV, PV_M, PV_V, PV_W, PV_H, PV_GIVENS, PV_Z = 1, 2, 4, 8, 16, 32, 64
PV_A_RESID, PV_B, PV_X, PV_AX = 128, 256, 512, 1024
PV_CORRECTION = PV_A_KRYLOV | PV_M | PV_V | PV_W | PV_H | PV_GIVENS | PV_Z
PV_REFINEMENT = PV_A_RESID | PV_B | PV_X | PV_AX

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


class Opts(ctypes.Structure):
    """Mirror of ``orc_opts`` (see gmres_oracle.h)."""

    _fields_ = [
        ("m", ctypes.c_int32),
        ("ortho", ctypes.c_int32),
        ("prec", ctypes.c_int32),
        ("maxiter", ctypes.c_int32),
        ("repeat_first", ctypes.c_int32),
        ("stall_window", ctypes.c_int32),
        ("tol", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("inner_factor", ctypes.c_double),
        ("stall_factor", ctypes.c_double),
        ("orth_threshold", ctypes.c_double),
        ("orth_norm", ctypes.c_int32),
        ("orth_iters", ctypes.c_int32),
        ("split_bytes", ctypes.c_int32),
        ("left_precond", ctypes.c_int32),
        ("ilu32", ctypes.c_int32),
        ("pv_mask", ctypes.c_int32),
    ]


class Restart(ctypes.Structure):
    """Mirror of ``orc_restart`` (see gmres_oracle.h)."""

    _fields_ = [
        ("tau", ctypes.c_double),
        ("inner_abs", ctypes.c_double),
        ("stall_factor", ctypes.c_double),
        ("orth_threshold", ctypes.c_double),
        ("stall_window", ctypes.c_int32),
        ("orth_norm", ctypes.c_int32),
        ("orth_iters", ctypes.c_int32),
        ("split_bytes", ctypes.c_int32),
        ("left_precond", ctypes.c_int32),
        ("ilu32", ctypes.c_int32),
        ("pv_mask", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    """Mirror of ``orc_info``."""

    _fields_ = [
        ("iters", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("first_len", ctypes.c_int32),
        ("relres", ctypes.c_double),
        ("bnorm", ctypes.c_double),
    ]


def _sources_present(src_dir=_HERE):
    return [os.path.join(src_dir, f) for f in _SOURCES if os.path.exists(os.path.join(src_dir, f))]


def build(force: bool = False, src_dir: str = _HERE, out_path: str = _LIB_PATH) -> str:
    """Compile the oracle sources in ``src_dir`` into ``out_path`` if missing or stale."""
    srcs = _sources_present(src_dir)
    newest = max(os.path.getmtime(f) for f in srcs)
    if force or not os.path.exists(out_path) or os.path.getmtime(out_path) < newest:
        c_files = [f for f in srcs if f.endswith(".c")]
        tmp = out_path + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp] + c_files + ["-lm"]
        subprocess.run(cmd, check=True, cwd=src_dir)
        os.replace(tmp, out_path)
    return out_path


_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_omp = None


def build_omp(force: bool = False) -> str:
    """The CPU-baseline timing build: the same sources with -O3 -fopenmp, so
    the loops over rows and vector entries run on every host core (the
    parity build above stays single-threaded and is the one tests use)."""
    srcs = _sources_present()
    newest = max(os.path.getmtime(f) for f in srcs)
    if force or not os.path.exists(_OMP_PATH) or os.path.getmtime(_OMP_PATH) < newest:
        c_files = [f for f in srcs if f.endswith(".c")]
        tmp = _OMP_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp] + c_files + ["-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _OMP_PATH)
    return _OMP_PATH


def lib_omp():
    """The OpenMP timing build, loaded (built on first use)."""
    global _omp
    with _lock:
        if _omp is None:
            build_omp()
            _omp = _bind(ctypes.CDLL(_OMP_PATH))
        return _omp


def _bind(L):
    L.orc_spmv.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int32]
    L.orc_spmv.restype = ctypes.c_int
    L.orc_residual.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p,
                               ctypes.c_void_p]
    L.orc_residual.restype = ctypes.c_double
    L.orc_round_basis.argtypes = [ctypes.c_int32, _f64p, _f64p, ctypes.c_int32, ctypes.c_int32]
    L.orc_round_basis.restype = None
    vp = ctypes.c_void_p
    L.orc_arnoldi_cycle.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                    vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                    ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32)]
    L.orc_arnoldi_cycle.restype = ctypes.c_int
    L.orc_arnoldi_cycle_ex.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.POINTER(Restart),
                                       vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]
    L.orc_arnoldi_cycle_ex.restype = ctypes.c_int
    L.orc_arnoldi_step.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, _f64p, _f64p]
    L.orc_arnoldi_step.restype = ctypes.c_int
    L.orc_s_norm2.argtypes = [ctypes.c_int32, _f64p, ctypes.c_int32, ctypes.c_int32]
    L.orc_s_norm2.restype = ctypes.c_double
    L.orc_high_part.argtypes = [ctypes.c_double]
    L.orc_high_part.restype = ctypes.c_double
    L.orc_ilu0.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p]
    L.orc_ilu0.restype = ctypes.c_int
    L.orc_ilu_apply.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.orc_ilu_apply.restype = ctypes.c_int
    L.orc_threads.argtypes = [ctypes.c_int32]
    L.orc_threads.restype = ctypes.c_int
    L.orc_gmres.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p,
                            ctypes.POINTER(Opts), vp, vp, vp, ctypes.POINTER(Info), vp, vp]
    L.orc_gmres.restype = ctypes.c_int
    if hasattr(L, "orc_spai_features"):
        _bind_spai(L)
    return L


def load_path(path):
    """Open an oracle build at ``path`` (used by the planted-mistake tests)."""
    return _bind(ctypes.CDLL(path))


def lib():
    """The loaded oracle library (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
        return _lib


_active = None  # when set, the wrappers below call this library instead of lib()


def _L():
    return _active if _active is not None else lib()


class use:
    """Context manager: route the module-level wrappers to another build."""

    def __init__(self, L):
        self.L = L

    def __enter__(self):
        global _active
        self.prev = _active
        _active = self.L
        return self.L

    def __exit__(self, *exc):
        global _active
        _active = self.prev
        return False


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(A):
    rowptr, colind, vals = A
    return (np.ascontiguousarray(rowptr, dtype=np.int32),
            np.ascontiguousarray(colind, dtype=np.int32),
            np.ascontiguousarray(vals, dtype=np.float64))


def spmv(A, x, prec=FP64):
    """y = A x (binary64, or binary32 values/sum for any other precision)."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    rc = _L().orc_spmv(n, rp, ci, va, x, y, prec)
    if rc:
        raise ValueError("orc_spmv failed: %d" % rc)
    return y


def residual(A, b, x):
    """(z, ||z||) with z = b - A x in binary64."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    z = np.empty(n, dtype=np.float64)
    nrm = _L().orc_residual(n, rp, ci, va, np.ascontiguousarray(b, np.float64),
                             np.ascontiguousarray(x, np.float64), _ptr(z))
    return z, nrm


def residual_norm(A, b, x):
    """||b - A x||_2 in binary64."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    return _L().orc_residual(n, rp, ci, va, np.ascontiguousarray(b, np.float64),
                              np.ascontiguousarray(x, np.float64), None)


def round_basis(v, prec, n):
    """Values a Krylov basis of precision ``prec`` stores for ``v`` (length-n system)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty_like(v)
    _L().orc_round_basis(v.size, v.ravel(), out.ravel(), prec, n)
    return out


def arnoldi_cycle(A, r0, m, ortho=CGSR, prec=FP64, kmax=None, tau=0.0, inner_abs=0.0, M=None,
                  export_basis=True, stall_factor=0.0, stall_window=0, orth_norm=ORTH_OFF,
                  orth_threshold=1.0, orth_iters=10, split_bytes=False, ilu=None,
                  ilu32=False, pv_mask=0):
    """One restart cycle from residual r0; returns a dict of its quantities.

    V is (m+1, n) (row i = basis vector i), Hbar/H are (m+1, m), the first ``j``
    columns valid.  ``export_basis=False`` skips copying V out (V is None).
    ``orth`` holds ||S_k|| after each inner iteration when ``orth_norm`` is
    set (third and fourth restart strategies of Sec. 3: stall_*, orth_*)."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    kmax = m if kmax is None else kmax
    V = np.zeros((m + 1, n)) if export_basis else None
    Hb = np.zeros((m, m + 1))
    H = np.zeros((m, m + 1))
    s = np.zeros(m + 1)
    cs = np.zeros(m)
    sn = np.zeros(m)
    y = np.zeros(m)
    u = np.zeros(n)
    arn = np.zeros(m)
    j = ctypes.c_int32(0)
    bd = ctypes.c_int32(0)
    rs = Restart()
    rs.tau, rs.inner_abs = tau, inner_abs
    rs.stall_factor = stall_factor
    rs.stall_window = stall_window if stall_window > 0 else (m + 19) // 20
    rs.orth_norm, rs.orth_threshold, rs.orth_iters = orth_norm, orth_threshold, orth_iters
    rs.split_bytes = int(bool(split_bytes))
    rs.pv_mask = int(pv_mask)
    if ilu is not None:
        if M is not None:
            raise ValueError("one preconditioner at a time")
        M = ilu
        rs.left_precond = 1
        rs.ilu32 = int(bool(ilu32))
    if M is not None:
        mp, mc, mv = _csr(M)
        keep = (mp, mc, mv)
        margs = (_ptr(mp), _ptr(mc), _ptr(mv))
    else:
        keep = None
        margs = (None, None, None)
    orth = np.zeros(m)
    rc = _L().orc_arnoldi_cycle_ex(n, rp, ci, va, np.ascontiguousarray(r0, np.float64), m, kmax,
                                    ortho, prec, ctypes.byref(rs), *margs, _ptr(V), _ptr(Hb),
                                    _ptr(H), _ptr(s), _ptr(cs), _ptr(sn), _ptr(y), _ptr(u),
                                    _ptr(arn), _ptr(orth), ctypes.byref(j), ctypes.byref(bd))
    del keep
    if rc:
        raise ValueError("orc_arnoldi_cycle failed: %d" % rc)
    jj = j.value
    return dict(V=V, Hbar=Hb.T.copy(), H=H.T.copy(), s=s, cs=cs, sn=sn, y=y, u=u, arn=arn, j=jj,
                breakdown=bool(bd.value), orth=orth)


def arnoldi_step(A, V, ortho=CGSR, prec=FP64):
    """One inner iteration from the basis V (rows = stored basis vectors):
    returns (h, vnext) with h = (h_{1..j,j}, h_{j+1,j}) and vnext = w / h_{j+1,j}
    in the working precision, before storage rounding."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, n)
    j = V.shape[0]
    h = np.zeros(j + 1)
    vnext = np.zeros(n)
    rc = _L().orc_arnoldi_step(n, rp, ci, va, V, j, ortho, prec, h, vnext)
    if rc:
        raise ValueError("orc_arnoldi_step failed: %d" % rc)
    return h, vnext


def ilu0(A):
    """ILU(0) factors of A on its pattern (Sec. 4's preconditioner): a CSR
    triple (rowptr, colind, lu) with L's strictly lower entries (unit
    diagonal implied) and U's upper entries including the diagonal."""
    rp, ci, va = _csr(A)
    lu = np.zeros(len(va))
    rc = _L().orc_ilu0(len(rp) - 1, rp, ci, va, lu)
    if rc:
        raise ValueError("orc_ilu0 failed: %d" % rc)
    return rp, ci, lu


def ilu_apply(LU, z):
    """(L U)^-1 z in binary64."""
    rp, ci, lu = _csr(LU)
    z = np.ascontiguousarray(z, dtype=np.float64)
    out = np.zeros(len(rp) - 1)
    rc = _L().orc_ilu_apply(len(rp) - 1, rp, ci, lu, z, out)
    if rc:
        raise ValueError("orc_ilu_apply failed: %d" % rc)
    return out


def threads(want=0):
    """Threads of the active build's row and vector loops (1 for the parity
    build); want > 0 sets them first (OpenMP timing build)."""
    return _L().orc_threads(int(want))


def high_part(v):
    """The high-order 32 bits of the binary64 value v, as a binary64 value."""
    return _L().orc_high_part(float(v))


def s_norm2(S, iters=10):
    """||S||_2 estimate of a strictly upper triangular S by the power method
    the fourth restart strategy uses (Sec. 3; 10 iterations in Sec. 4.1)."""
    S = np.asfortranarray(S, dtype=np.float64)
    k = S.shape[0]
    return _L().orc_s_norm2(k, S.ravel(order="F"), k, iters)


def default_tau(prec):
    """Restart threshold on the Arnoldi-residual gain per precision (Sec. 3,
    second strategy): the performance study's 1e-6 for binary32; for the
    16-bit bases one unit roundoff of the storage format (2^-8, 2^-11)."""
    return {FP64: 0.0, MIXED: 1e-6, MIXED_BF16: 2.0 ** -8, MIXED_FP16: 2.0 ** -11,
            ALL_FP32: 1e-6, MIXED_LIMITED: 1e-6}[prec]


def gmres(A, b, x0=None, m=30, tol=1e-10, ortho=CGSR, prec=FP64, maxiter=10000, tau=None,
          repeat_first=None, inner_factor=0.5, M=None, history=False, stall_factor=0.0,
          stall_window=0, orth_norm=ORTH_OFF, orth_threshold=1.0, orth_iters=10,
          split_bytes=False, ilu=None, ilu32=False, pv_mask=0):
    """Restarted GMRES(m) (Algorithm 1).  Returns (x, info dict).

    Restart strategies (Sec. 3): repeat_first (first), tau (second),
    stall_factor/stall_window (third; window 0 = ceil(0.05 m)), orth_norm /
    orth_threshold / orth_iters (fourth, loss of orthogonality via ||S_k||).
    split_bytes: A stored as high/low 32-bit halves, the Krylov step reading
    the high-order half (Sec. 4).  pv_mask: PV_* bits, the per-variable
    precision study of Sec. 4.1 (with prec=FP64)."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    o = Opts()
    o.m, o.ortho, o.prec, o.maxiter = m, ortho, prec, maxiter
    o.repeat_first = int(prec != FP64) if repeat_first is None else int(repeat_first)
    o.tol = tol
    o.tau = default_tau(prec) if tau is None else tau
    o.inner_factor = inner_factor
    o.stall_factor, o.stall_window = stall_factor, stall_window
    o.orth_norm, o.orth_threshold, o.orth_iters = orth_norm, orth_threshold, orth_iters
    o.split_bytes = int(bool(split_bytes))
    o.pv_mask = int(pv_mask)
    if ilu is not None:
        if M is not None:
            raise ValueError("one preconditioner at a time")
        M = ilu
        o.left_precond = 1
        o.ilu32 = int(bool(ilu32))
    info = Info()
    arn = np.zeros(max(maxiter, 1)) if history else None
    cyc = np.zeros(maxiter + 2) if history else None
    if M is not None:
        mp, mc, mv = _csr(M)
        margs = (_ptr(mp), _ptr(mc), _ptr(mv))
    else:
        mp = mc = mv = None
        margs = (None, None, None)
    rc = _L().orc_gmres(n, rp, ci, va, b, x, ctypes.byref(o), *margs, ctypes.byref(info),
                         _ptr(arn), _ptr(cyc))
    if rc:
        raise ValueError("orc_gmres failed: %d" % rc)
    out = dict(iters=info.iters, restarts=info.restarts, converged=bool(info.converged),
               first_len=info.first_len, relres=info.relres, bnorm=info.bnorm)
    if history:
        out["arnoldi"] = arn[: info.iters].copy()
        out["cycle_relres"] = cyc[: info.restarts + 1].copy()
    return x, out


def _bind_spai(L):
    i64 = ctypes.c_int64
    vp = ctypes.c_void_p
    L.orc_spai_nparam.argtypes = []
    L.orc_spai_nparam.restype = ctypes.c_int
    L.orc_spai_features.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p]
    L.orc_spai_features.restype = ctypes.c_int
    L.orc_spai_forward.argtypes = [i64, _f64p, _f64p, _f64p]
    L.orc_spai_forward.restype = ctypes.c_int
    L.orc_spai_values.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
    L.orc_spai_values.restype = ctypes.c_int
    L.orc_spai_loss_grad_m.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p,
                                       ctypes.c_int32, _f64p, vp]
    L.orc_spai_loss_grad_m.restype = ctypes.c_double
    L.orc_spai_loss_grad.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, ctypes.c_int32,
                                     _f64p, vp, vp]
    L.orc_spai_loss_grad.restype = ctypes.c_double
    L.orc_adam_step.argtypes = [ctypes.c_int32, _f64p, _f64p, _f64p, _f64p, ctypes.c_int32,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double]
    L.orc_adam_step.restype = None


SPAI_NF, SPAI_NH = 8, 64
SPAI_NPARAM = SPAI_NH * SPAI_NF + SPAI_NH + SPAI_NH * SPAI_NH + SPAI_NH + SPAI_NH + 1


def spai_unpack(params):
    """(W1[64,8], b1[64], W2[64,64], b2[64], w3[64], b3) views of a parameter vector."""
    p = np.asarray(params)
    o = 0
    W1 = p[o:o + 512].reshape(64, 8); o += 512
    b1 = p[o:o + 64]; o += 64
    W2 = p[o:o + 4096].reshape(64, 64); o += 4096
    b2 = p[o:o + 64]; o += 64
    w3 = p[o:o + 64]; o += 64
    return W1, b1, W2, b2, w3, p[o]


def spai_jacobi_params():
    """Parameters whose network outputs g = [p == q] exactly, i.e. M = D^-1."""
    p = np.zeros(SPAI_NPARAM)
    W1, b1, W2, b2, w3, _ = spai_unpack(p)
    W1[0, 2] = 1.0
    W2[0, 0] = 1.0
    w3[0] = 1.0
    return p


def spai_features(A):
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    f = np.zeros((len(ci), 8))
    _L().orc_spai_features(n, rp, ci, va, f)
    return f


def spai_forward(feat, params):
    feat = np.ascontiguousarray(feat, np.float64)
    g = np.zeros(feat.shape[0])
    _L().orc_spai_forward(feat.shape[0], feat, np.ascontiguousarray(params, np.float64), g)
    return g


def spai_values(A, params):
    rp, ci, va = _csr(A)
    m = np.zeros(len(ci))
    _L().orc_spai_values(len(rp) - 1, rp, ci, va, np.ascontiguousarray(params, np.float64), m)
    return m


def spai_loss_grad_m(A, mvals, Z, grad=True):
    """(loss, dL/dm) for M's values on A's pattern; Z is (P, n)."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    Z = np.ascontiguousarray(Z, np.float64).reshape(-1, n)
    g = np.zeros(len(ci)) if grad else None
    loss = _L().orc_spai_loss_grad_m(n, rp, ci, va, np.ascontiguousarray(mvals, np.float64),
                                     Z.shape[0], Z, _ptr(g))
    return loss, g


def spai_loss_grad(A, params, Z, grad=True):
    """(loss, dL/dparams, dL/dm) of the learned preconditioner; Z is (P, n)."""
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    Z = np.ascontiguousarray(Z, np.float64).reshape(-1, n)
    gp = np.zeros(SPAI_NPARAM) if grad else None
    gm = np.zeros(len(ci)) if grad else None
    loss = _L().orc_spai_loss_grad(n, rp, ci, va, np.ascontiguousarray(params, np.float64),
                                   Z.shape[0], Z, _ptr(gp), _ptr(gm))
    return loss, gp, gm


def adam_step(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in binary64 on copies; returns (p, m, v)."""
    p = np.array(p, dtype=np.float64)
    m = np.array(m, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    _L().orc_adam_step(p.size, p, m, v, np.ascontiguousarray(g, np.float64), t, lr, b1, b2, eps)
    return p, m, v

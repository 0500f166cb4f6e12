"""ctypes binding of libgmres_gb300.so (C-ABI in include/gmres_gb300.h).

Argument marshalling only: every entry point forwards to the CUDA library
under the same name.  Arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA memory); their data pointers are passed through
unchanged.  There is no CPU implementation behind this module: when the
shared library is missing it raises instead of computing anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# GMRES_GB300_CHECKS=1 in the environment loads the checked build instead
# (column indices tested in the kernels; gmres_checks_enabled)
CHECKED = os.environ.get("GMRES_GB300_CHECKS") == "1"
LIB_PATH = _build.LIB_CHECKED_PATH if CHECKED else _build.LIB_PATH

# enums (include/gmres_gb300.h)
ORTHO_MGS, ORTHO_CGSR = 0, 1
FP64, MIXED, MIXED_BF16, MIXED_FP16, MIXED_LIMITED = 0, 1, 2, 3, 4
OK, MAXITER, ERR_ARG, ERR_CUDA, ERR_NONFINITE, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_OOM = (
    0, 1, -1, -2, -3, -4, -5, -6)
ERR_INDEX = -7
CREATE_DEVICE_PTRS, CREATE_TRANSPOSE, CREATE_SPLIT = 1, 2, 4
PATH_AUTO, PATH_GRID, PATH_BLOCK = 0, 1, 2
PRECOND_NONE, PRECOND_SPAI, PRECOND_ILU0 = 0, 1, 2
ORTH_OFF, ORTH_SPECTRAL, ORTH_FROBENIUS = 0, 1, 2
# per-variable precision switches (gmres_opts.pv_mask)
PV_A_KRYLOV, PV_M, PV_V, PV_W, PV_H, PV_GIVENS, PV_Z = 1, 2, 4, 8, 16, 32, 64
PV_A_RESID, PV_B, PV_X, PV_AX = 128, 256, 512, 1024
# storage of A for the Krylov step's product (gmres_opts.spmv_format)
SPMV_AUTO, SPMV_CSR, SPMV_SLICED = 0, 1, 2
K_RESIDUAL, K_SPMV, K_ORTHO, K_NORMALIZE, K_UPDATE, K_PRECOND, K_BLOCK = range(7)
K_COUNT = 8
KERNEL_CLASS_NAMES = ["residual", "spmv", "ortho", "normalize", "update", "precond", "block"]

PRECISIONS = {"fp64": FP64, "mixed": MIXED, "mixed_bf16": MIXED_BF16, "mixed_fp16": MIXED_FP16,
              "mixed_limited": MIXED_LIMITED}
ORTHOS = {"mgs": ORTHO_MGS, "cgsr": ORTHO_CGSR}


class GmresError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, status_str(status), status))


class Opts(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double),
        ("inner_factor", ctypes.c_double),
        ("repeat_first", ctypes.c_int32),
        ("path", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("spin_limit", ctypes.c_int32),
        ("precond", ctypes.c_int32),
        ("fallback", ctypes.c_int32),
        ("spmv_lanes", ctypes.c_int32),
        ("cgs_kernel", ctypes.c_int32),
        ("mgs_kernel", ctypes.c_int32),
        ("l2_prefetch", ctypes.c_int32),
        ("block_cluster", ctypes.c_int32),
        ("ilu_binary32", ctypes.c_int32),
        ("stall_factor", ctypes.c_double),
        ("stall_window", ctypes.c_int32),
        ("orth_norm", ctypes.c_int32),
        ("orth_threshold", ctypes.c_double),
        ("orth_iters", ctypes.c_int32),
        ("trsv_kernel", ctypes.c_int32),
        ("pv_mask", ctypes.c_int32),
        ("spmv_format", ctypes.c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("restarts", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("first_len", ctypes.c_int32),
        ("relres", ctypes.c_double),
        ("bnorm", ctypes.c_double),
        ("time_ms", ctypes.c_double),
        ("kernel_ms", ctypes.c_double * K_COUNT),
        ("kernel_bytes", ctypes.c_double * K_COUNT),
        ("kernel_launches", ctypes.c_int64 * K_COUNT),
        ("launches", ctypes.c_int64),
        ("path", ctypes.c_int32),
        ("fell_back", ctypes.c_int32),
    ]

    def as_dict(self):
        return dict(
            iters=self.iters, restarts=self.restarts, converged=bool(self.converged),
            first_len=self.first_len, relres=self.relres, bnorm=self.bnorm,
            time_ms=self.time_ms, launches=self.launches, path=self.path,
            fell_back=bool(self.fell_back),
            kernel_ms={KERNEL_CLASS_NAMES[i]: self.kernel_ms[i] for i in range(7)},
            kernel_bytes={KERNEL_CLASS_NAMES[i]: self.kernel_bytes[i] for i in range(7)},
            kernel_launches={KERNEL_CLASS_NAMES[i]: self.kernel_launches[i] for i in range(7)},
        )


# Every exported symbol of the C-ABI with its ctypes signature.
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_f64 = ctypes.c_double
_st = ctypes.c_int
SIGNATURES = {
    "gmres_default_opts": (None, [ctypes.POINTER(Opts)]),
    "gmres_create": (_st, [ctypes.POINTER(_vp), _i32, _vp, _vp, _vp, _i32, _vp]),
    "gmres_destroy": (None, [_vp]),
    "gmres_set_stream": (_st, [_vp, _vp]),
    "gmres_set_opts": (_st, [_vp, ctypes.POINTER(Opts)]),
    "gmres_get_opts": (_st, [_vp, ctypes.POINTER(Opts)]),
    "gmres_solve": (_st, [_vp, _vp, _vp, _i32, _f64, _i32, _i32, _i32, ctypes.POINTER(Info)]),
    "gmres_spmv": (_st, [_vp, _vp, _vp, _i32]),
    "gmres_residual": (_st, [_vp, _vp, _vp, _vp, ctypes.POINTER(_f64)]),
    "gmres_arnoldi": (_st, [_vp, _vp, _i32, _i32, _i32, _i32, _f64, _f64] + [_vp] * 9
                      + [ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "gmres_arnoldi_step": (_st, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "gmres_autotune": (_st, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "gmres_spmv_format": (_st, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "gmres_checks_enabled": (_i32, []),
    "gmres_memory_bytes": (_st, [_vp, _i32, _i32, ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(ctypes.c_int64)]),
    "gmres_orth_norms": (_st, [_vp, _vp, _i32]),
    "gmres_backward_error": (_st, [_vp, _vp, _vp, ctypes.POINTER(_f64)]),
    "gmres_ilu0": (_st, [_vp]),
    "gmres_ilu_apply": (_st, [_vp, _vp, _vp, _i32]),
    "gmres_ilu_factors": (_st, [_vp, _vp]),
    "gmres_ilu_levels": (_st, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "gmres_batch_autotune": (_st, [_vp, _vp, _i32, _i32, _i32, _i32, ctypes.POINTER(_i32)]),
    "gmres_batch_set_cluster_rows": (_st, [_vp, _i32]),
    "gmres_batch_set_cluster_threads": (_st, [_vp, _i32]),
    "gmres_batch_create": (_st, [ctypes.POINTER(_vp), _i32, _vp, _vp, _vp, _vp, _vp]),
    "gmres_batch_destroy": (None, [_vp]),
    "gmres_batch_solve": (_st, [_vp, _vp, _vp, _i32, _f64, _i32, _i32, _i32, _i32, _vp,
                                ctypes.POINTER(Info)]),
    "gmres_set_values": (_st, [_vp, _vp]),
    "gmres_spai_features": (_st, [_vp, _vp]),
    "gmres_spai_loss_grad": (_st, [_vp, _vp, _i32, _vp, ctypes.POINTER(_f64), _vp, _vp]),
    "gmres_spai_adam": (_st, [_vp, _vp, _vp, _vp, _vp, _i32, ctypes.c_float]),
    "gmres_spai_train_step": (_st, [_vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_uint64, _vp, _i32,
                                    ctypes.c_float, ctypes.POINTER(_f64)]),
    "gmres_spai_set": (_st, [_vp, _vp]),
    "gmres_spai_values": (_st, [_vp, _vp]),
    "gmres_spai_clear": (_st, [_vp]),
    "gmres_solve_noalloc": (_st, [_i32, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _i32, _f64,
                                  _i32, _i32, _i32, _vp, ctypes.POINTER(Info)]),
    "gmres_status_str": (ctypes.c_char_p, [_st]),
    "gmres_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """Load libgmres_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is missing: run paper_2011_01850_gb300.build "
                               "(or __graft_entry__.build()) first; there is no fallback"
                               % os.path.basename(LIB_PATH))
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_str(s):
    try:
        return lib().gmres_status_str(int(s)).decode()
    except Exception:  # library not loadable: still give a readable message
        return "status %d" % s


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError("unsupported array type %r" % type(a))


def _check(st, where):
    if st < 0:
        raise GmresError(st, where)
    return st


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ----------------------------------------------------------------------------
# same-named wrappers
# ----------------------------------------------------------------------------

def gmres_default_opts():
    o = Opts()
    lib().gmres_default_opts(ctypes.byref(o))
    return o


def gmres_create(n, rowptr, colind, vals, flags=0, stream=None):
    h = ctypes.c_void_p()
    st = lib().gmres_create(ctypes.byref(h), int(n), _ptr(rowptr), _ptr(colind), _ptr(vals),
                            int(flags), _stream_ptr(stream))
    _check(st, "gmres_create")
    return h


def gmres_destroy(h):
    lib().gmres_destroy(h)


def gmres_set_stream(h, stream):
    return _check(lib().gmres_set_stream(h, _stream_ptr(stream)), "gmres_set_stream")


def gmres_set_opts(h, opts):
    return _check(lib().gmres_set_opts(h, ctypes.byref(opts)), "gmres_set_opts")


def gmres_get_opts(h):
    o = Opts()
    _check(lib().gmres_get_opts(h, ctypes.byref(o)), "gmres_get_opts")
    return o


def gmres_solve(h, b, x, m, tol, ortho, prec, maxiter):
    """Returns (status, Info).  Negative statuses raise GmresError."""
    info = Info()
    st = lib().gmres_solve(h, _ptr(b), _ptr(x), int(m), float(tol), int(ortho), int(prec),
                           int(maxiter), ctypes.byref(info))
    _check(st, "gmres_solve")
    return st, info


def gmres_spmv(h, x, y, prec):
    return _check(lib().gmres_spmv(h, _ptr(x), _ptr(y), int(prec)), "gmres_spmv")


def gmres_residual(h, b, x, z=None):
    nrm = ctypes.c_double()
    _check(lib().gmres_residual(h, _ptr(b), _ptr(x), _ptr(z), ctypes.byref(nrm)),
           "gmres_residual")
    return nrm.value


def gmres_arnoldi(h, r0, m, kmax, ortho, prec, tau=0.0, inner_abs=0.0, n=None):
    """One restart cycle; returns a dict shaped like oracle.arnoldi_cycle."""
    n = int(n if n is not None else r0.shape[0])
    V = np.zeros((m + 1, n))
    Hb = np.zeros((m, m + 1))
    H = np.zeros((m, m + 1))
    s = np.zeros(m + 1)
    cs = np.zeros(m)
    sn = np.zeros(m)
    y = np.zeros(m)
    u = np.zeros(n)
    arn = np.zeros(m)
    j = ctypes.c_int32()
    bd = ctypes.c_int32()
    st = lib().gmres_arnoldi(h, _ptr(r0), int(m), int(kmax), int(ortho), int(prec), float(tau),
                             float(inner_abs), _ptr(V), _ptr(Hb), _ptr(H), _ptr(s), _ptr(cs),
                             _ptr(sn), _ptr(y), _ptr(u), _ptr(arn), ctypes.byref(j),
                             ctypes.byref(bd))
    _check(st, "gmres_arnoldi")
    return dict(V=V, Hbar=Hb.T.copy(), H=H.T.copy(), s=s, cs=cs, sn=sn, y=y, u=u, arn=arn,
                j=j.value, breakdown=bool(bd.value))


def gmres_arnoldi_step(h, V, ortho, prec, want_v=True):
    """One inner iteration from the basis V (rows = basis vectors, host
    binary64): returns (hcol, vnext) with hcol = (h_{1..j,j}, h_{j+1,j})."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    ncols, n = V.shape
    hcol = np.zeros(ncols + 1)
    vnext = np.zeros(n) if want_v else None
    st = lib().gmres_arnoldi_step(h, _ptr(V), int(ncols), int(ortho), int(prec), _ptr(hcol),
                                  _ptr(vnext))
    _check(st, "gmres_arnoldi_step")
    return hcol, vnext


def gmres_autotune(h):
    a = ctypes.c_int32()
    b = ctypes.c_int32()
    _check(lib().gmres_autotune(h, ctypes.byref(a), ctypes.byref(b)), "gmres_autotune")
    return a.value, b.value


def gmres_checks_enabled():
    """1 when the loaded library is the checked build (GMRES_GB300_CHECKS=1)."""
    return int(lib().gmres_checks_enabled())


def gmres_spmv_format(h):
    """(binary32, binary64) storage of A the product reads: SPMV_CSR or
    SPMV_SLICED."""
    a = ctypes.c_int32()
    b = ctypes.c_int32()
    _check(lib().gmres_spmv_format(h, ctypes.byref(a), ctypes.byref(b)), "gmres_spmv_format")
    return a.value, b.value


def gmres_batch_set_cluster_rows(h, min_rows):
    """Systems of at least min_rows rows go to 8-block clusters (0: none)."""
    return _check(lib().gmres_batch_set_cluster_rows(h, int(min_rows)),
                  "gmres_batch_set_cluster_rows")

def gmres_batch_set_cluster_threads(h, threads):
    """Threads per block of the clusters that solve the large systems."""
    return _check(lib().gmres_batch_set_cluster_threads(h, int(threads)),
                  "gmres_batch_set_cluster_threads")


def gmres_batch_autotune(h, rhs, m, ortho, prec, iters):
    """Time capped batched solves over the SpMV lanes candidates; returns
    the lanes per row the batch keeps for lanes = 0."""
    out = _i32()
    _check(lib().gmres_batch_autotune(h, _ptr(rhs), int(m), int(ortho), int(prec), int(iters),
                                      ctypes.byref(out)), "gmres_batch_autotune")
    return out.value


def gmres_ilu0(h):
    """ILU(0) factors of the handle's matrix (select with precond=2)."""
    return _check(lib().gmres_ilu0(h), "gmres_ilu0")


def gmres_ilu_levels(h):
    """(levels of L, levels of U) of the ILU(0) factors."""
    lo, up = _i32(), _i32()
    _check(lib().gmres_ilu_levels(h, ctypes.byref(lo), ctypes.byref(up)), "gmres_ilu_levels")
    return lo.value, up.value


def gmres_ilu_factors(h, nnz):
    """The binary64 ILU(0) factors on A's pattern (host array)."""
    lu = np.zeros(int(nnz))
    _check(lib().gmres_ilu_factors(h, lu.ctypes.data_as(_vp)), "gmres_ilu_factors")
    return lu


def gmres_ilu_apply(h, z, out, prec):
    """out = (L U)^-1 z on the device."""
    return _check(lib().gmres_ilu_apply(h, _ptr(z), _ptr(out), int(prec)), "gmres_ilu_apply")


def gmres_backward_error(h, b, x):
    """||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) for device b, x."""
    eta = _f64()
    _check(lib().gmres_backward_error(h, _ptr(b), _ptr(x), ctypes.byref(eta)),
           "gmres_backward_error")
    return eta.value


def gmres_orth_norms(h, count):
    """||S_k|| after each inner iteration of the handle's last cycle."""
    out = np.zeros(int(count))
    _check(lib().gmres_orth_norms(h, out.ctypes.data_as(_vp), int(count)), "gmres_orth_norms")
    return out


def gmres_memory_bytes(h, m, prec):
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    _check(lib().gmres_memory_bytes(h, int(m), int(prec), ctypes.byref(a), ctypes.byref(b)),
           "gmres_memory_bytes")
    return a.value, b.value


SPAI_NPARAM = 4801


def gmres_set_values(h, vals):
    return _check(lib().gmres_set_values(h, _ptr(vals)), "gmres_set_values")


def gmres_spai_features(h, feat=None):
    return _check(lib().gmres_spai_features(h, _ptr(feat)), "gmres_spai_features")


def gmres_spai_loss_grad(h, params, nprobe, Z, grad_params=None, grad_m=None):
    loss = ctypes.c_double()
    _check(lib().gmres_spai_loss_grad(h, _ptr(params), int(nprobe), _ptr(Z), ctypes.byref(loss),
                                      _ptr(grad_params), _ptr(grad_m)), "gmres_spai_loss_grad")
    return loss.value


def gmres_spai_adam(h, params, adam_m, adam_v, grad, step, lr):
    return _check(lib().gmres_spai_adam(h, _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(grad),
                                        int(step), float(lr)), "gmres_spai_adam")


def gmres_spai_train_step(h, params, adam_m, adam_v, step, nprobe, seed, Zx=None, nzx=0, lr=1e-3):
    loss = ctypes.c_double()
    _check(lib().gmres_spai_train_step(h, _ptr(params), _ptr(adam_m), _ptr(adam_v), int(step),
                                       int(nprobe), int(seed) & ((1 << 64) - 1), _ptr(Zx),
                                       int(nzx), float(lr), ctypes.byref(loss)),
           "gmres_spai_train_step")
    return loss.value


def gmres_spai_set(h, params):
    return _check(lib().gmres_spai_set(h, _ptr(params)), "gmres_spai_set")


def gmres_spai_values(h, mvals):
    return _check(lib().gmres_spai_values(h, _ptr(mvals)), "gmres_spai_values")


def gmres_spai_clear(h):
    return _check(lib().gmres_spai_clear(h), "gmres_spai_clear")


class BatchResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("relres", ctypes.c_double)]


def gmres_batch_create(nsys, sys_ptr, rowptr, colind, vals, stream=None):
    h = ctypes.c_void_p()
    st = lib().gmres_batch_create(ctypes.byref(h), int(nsys), _ptr(sys_ptr), _ptr(rowptr),
                                  _ptr(colind), _ptr(vals), _stream_ptr(stream))
    _check(st, "gmres_batch_create")
    return h


def gmres_batch_destroy(h):
    lib().gmres_batch_destroy(h)


def gmres_batch_solve(h, b, x, m, tol, ortho, prec, maxiter, lanes=0, nsys=None):
    """Returns (status, per-system results array, Info)."""
    res = (BatchResult * nsys)() if nsys else None
    info = Info()
    st = lib().gmres_batch_solve(h, _ptr(b), _ptr(x), int(m), float(tol), int(ortho), int(prec),
                                 int(maxiter), int(lanes),
                                 ctypes.cast(res, ctypes.c_void_p) if res is not None else None,
                                 ctypes.byref(info))
    _check(st, "gmres_batch_solve")
    return st, res, info


def pack_batch(systems):
    """Block-diagonal CSR of [(A_i, b_i), ...]: (sys_ptr, rowptr, colind, vals, b)."""
    sys_ptr = [0]
    rps, cis, vas, bs = [], [], [], []
    nnz0 = 0
    for A, b in systems:
        rp, ci, va = A
        n = len(rp) - 1
        rps.append(np.asarray(rp[:-1], np.int64) + nnz0)
        cis.append(np.asarray(ci, np.int64) + sys_ptr[-1])
        vas.append(np.asarray(va, np.float64))
        bs.append(np.asarray(b, np.float64))
        nnz0 += int(rp[-1])
        sys_ptr.append(sys_ptr[-1] + n)
    rowptr = np.concatenate(rps + [np.array([nnz0])]).astype(np.int32)
    return (np.array(sys_ptr, np.int64), rowptr, np.concatenate(cis).astype(np.int32),
            np.concatenate(vas), np.concatenate(bs))


NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def gmres_solve_noalloc(n, rowptr, colind, vals, nnz, b, x, m, tol, ortho, prec, maxiter,
                        stream=None):
    """Solve on caller-owned device arrays with no device allocation.
    Returns (status, Info); negative statuses raise GmresError."""
    info = Info()
    st = lib().gmres_solve_noalloc(int(n), _ptr(rowptr), _ptr(colind), _ptr(vals), int(nnz),
                                   _ptr(b), _ptr(x), int(m), float(tol), int(ortho), int(prec),
                                   int(maxiter), _stream_ptr(stream), ctypes.byref(info))
    _check(st, "gmres_solve_noalloc")
    return st, info


def gmres_status_str(s):
    return status_str(s)


def gmres_version():
    return lib().gmres_version().decode()


# ----------------------------------------------------------------------------
# convenience: a handle that owns its matrix
# ----------------------------------------------------------------------------

class Solver:
    """RAII wrapper around a gmres handle for a CSR matrix (numpy arrays)."""

    def __init__(self, A, flags=0, stream=None):
        rowptr, colind, vals = A
        self._keep = (np.ascontiguousarray(rowptr, dtype=np.int32),
                      np.ascontiguousarray(colind, dtype=np.int32),
                      np.ascontiguousarray(vals, dtype=np.float64))
        self.n = len(self._keep[0]) - 1
        self.h = gmres_create(self.n, *self._keep, flags=flags, stream=stream)

    def set_opts(self, **kw):
        o = gmres_get_opts(self.h)
        for k, v in kw.items():
            setattr(o, k, v)
        gmres_set_opts(self.h, o)

    def solve(self, b, x=None, m=30, tol=1e-10, ortho="cgsr", prec="mixed", maxiter=10000):
        if isinstance(ortho, str):
            ortho = ORTHOS[ortho]
        if isinstance(prec, str):
            prec = PRECISIONS[prec]
        if x is None:
            x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.new_zeros(self.n)
        st, info = gmres_solve(self.h, b, x, m, tol, ortho, prec, maxiter)
        return x, st, info.as_dict()

    def close(self):
        if self.h:
            gmres_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

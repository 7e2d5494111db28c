"""Python binding of ``libesdcg`` (include/esdcg.h): deflated / subspace-corrected ICCG for a
sequence of SPD systems with one matrix, the auxiliary matrix built from sampled error
vectors (arXiv 2203.08498).

Argument marshalling only: every numerical step runs in the library's CUDA kernels. Arrays
may be CUDA torch tensors, CPU torch tensors or NumPy arrays (host data is staged by the
library). There is no fallback: without the compiled library every call raises.

The functions keep the C names (``esd_create_matrix``, ``esd_solve`` ...); ``Matrix`` and
``Solver`` own the handles. A sequence as the paper runs it::

    A = Matrix(rowptr, colind, val, colour_ptr)        # CSR in multicolour order
    A.factor_ic0()                                     # IC(0), M = L L^T
    S = Solver(A, sample_cap=16)
    S.solve(b1, x1, tol=1e-8, sample_m=16)             # plain ICCG, 16 iterates sampled
    S.sample_and_build_W()                             # W from the error vectors, E = W^T A W
    S.set_mode(DEFLATION)                              # or SUBSPACE_CORRECTION
    for b, x in later_systems:
        status, iters, relres = S.solve(b, x, tol=1e-8)

Options: ``Solver(..., precision=FP32_REFINE)`` (FP32 inner PCG in FP64 refinement),
``sampling=SAMPLING_B``, ``power_start`` / ``paper_cond_estimate`` (the paper's condition
estimate), ``set_precond_matrix`` (block-Jacobi IC), ``Matrix(..., diag_scale=True)``;
``adjoint.fv_solve`` differentiates a solve through the adjoint.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import _build

__all__ = [
    "lib", "EsdError", "Matrix", "Solver", "PLAIN", "DEFLATION", "SUBSPACE_CORRECTION",
    "PRECOND_NONE", "PRECOND_IC0", "FP64", "FP32_REFINE", "SAMPLING_A", "SAMPLING_B", "EsdParams", "HEADER_SYMBOLS",
    "esd_create_matrix", "esd_matrix_destroy", "esd_matrix_info", "esd_matrix_layout", "esd_factor_ic0",
    "esd_matrix_spmv",
    "esd_matrix_apply_ic", "esd_pattern_grad", "esd_params_default", "esd_solver_create",
    "esd_solver_destroy", "esd_set_mode", "esd_solve", "esd_solve_pair", "esd_true_relres", "esd_last_solve_info",
    "esd_sample_and_build_W",
    "esd_set_W", "esd_get_W", "esd_ritz_values", "esd_estimate_cond", "esd_get_history",
    "esd_get_samples", "esd_backward_euler_rhs", "esd_profile_iterations", "esd_profile_pair_iterations",
    "esd_last_error",
    "esd_lanczos_extremes_noalloc", "NOALLOC_MAX_K", "esd_matrix_set_values", "esd_fv_assemble",
    "esd_fv_grad_theta", "esd_refresh_W", "EsdFvGrid", "esd_power_start", "esd_power_estimate",
    "esd_matrix_diag_scale", "MATRIX_DIAG_SCALE", "esd_set_precision", "esd_solver_set_precond_matrix",
    "esd_paper_cond_estimate",
]
MATRIX_DIAG_SCALE = 1
NOALLOC_MAX_K = 32768

OK, ERR_INVALID, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_MAXIT, ERR_STATE, ERR_RANK, ERR_CHOL_E, ERR_CUDA, ERR_NOMEM = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9)
ERR_INTERNAL = -10
PLAIN, DEFLATION, SUBSPACE_CORRECTION = 0, 1, 2
PRECOND_NONE, PRECOND_IC0 = 0, 1
FP64, FP32_REFINE = 0, 1
SAMPLING_A, SAMPLING_B = 0, 1

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "esdcg.h")


def _header_symbols():
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(esd_[a-zA-Z0-9_]+)\s*\(", txt)))


HEADER_SYMBOLS = _header_symbols()


class EsdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class EsdFvGrid(C.Structure):
    _fields_ = [("dims", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("h", C.c_double), ("inv_dt", C.c_double)]


class EsdParams(C.Structure):
    _fields_ = [("precond", C.c_int32), ("maxit_cap", C.c_int32), ("sample_cap", C.c_int32),
                ("lmax", C.c_int32), ("rank_tol", C.c_double), ("precision", C.c_int32),
                ("inner_tol", C.c_double), ("max_outer", C.c_int32), ("resume_direction", C.c_int32),
                ("sampling", C.c_int32)]


_lib = None


def lib(build_if_missing: bool = True):
    """Load the compiled library (building it in-tree when it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise EsdError(ERR_INVALID, f"libesdcg not built ({path})")
        L = C.CDLL(path)
        vp, i32, i64, f64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint32
        P = C.POINTER
        sig = {
            "esd_last_error": (C.c_char_p, []),
            "esd_create_matrix": (i32, [i32, i64, vp, vp, vp, vp, i32, u32, vp, P(vp)]),
            "esd_matrix_destroy": (i32, [vp]),
            "esd_matrix_info": (i32, [vp, P(i32), P(i64), P(i32), P(i32), P(i32)]),
            "esd_matrix_layout": (i32, [vp, P(i32), P(i64), P(i32)]),
            "esd_factor_ic0": (i32, [vp, i32, P(f64)]),
            "esd_matrix_spmv": (i32, [vp, vp, vp]),
            "esd_matrix_apply_ic": (i32, [vp, vp, vp]),
            "esd_pattern_grad": (i32, [vp, vp, vp, vp]),
            "esd_params_default": (None, [P(EsdParams)]),
            "esd_solver_create": (i32, [vp, P(EsdParams), P(vp)]),
            "esd_solver_destroy": (i32, [vp]),
            "esd_set_mode": (i32, [vp, i32]),
            "esd_solve": (i32, [vp, vp, vp, f64, i32, i32, P(i32), P(f64)]),
            "esd_solve_pair": (i32, [vp, vp, vp, vp, vp, vp, f64, i32, P(i32), P(f64), P(i32), P(f64), P(i32)]),
            "esd_true_relres": (i32, [vp, P(f64)]),
            "esd_last_solve_info": (i32, [vp, P(i32), P(i32), P(i32), P(i32), P(f64), P(f64), P(i32)]),
            "esd_sample_and_build_W": (i32, [vp, f64, P(i32)]),
            "esd_set_W": (i32, [vp, vp, i32]),
            "esd_get_W": (i32, [vp, vp, vp, vp, P(i32)]),
            "esd_ritz_values": (i32, [vp, vp, i32, P(i32)]),
            "esd_estimate_cond": (i32, [vp, P(f64), P(f64), P(f64), P(f64)]),
            "esd_get_history": (i32, [vp, vp, vp, i32, P(i32)]),
            "esd_get_samples": (i32, [vp, vp, vp, i32, P(i32)]),
            "esd_backward_euler_rhs": (i32, [vp, vp, vp, f64, vp]),
            "esd_profile_iterations": (i32, [vp, vp, vp, i32, vp, vp, i32, P(i32)]),
            "esd_profile_pair_iterations": (i32, [vp, vp, vp, vp, vp, vp, i32, vp, vp, i32, P(i32)]),
            "esd_lanczos_extremes_noalloc": (i32, [vp, vp, i32, vp, vp]),
            "esd_matrix_set_values": (i32, [vp, vp]),
            "esd_fv_assemble": (i32, [vp, P(EsdFvGrid), vp, vp]),
            "esd_fv_grad_theta": (i32, [vp, P(EsdFvGrid), vp, vp, vp, vp, vp]),
            "esd_refresh_W": (i32, [vp]),
            "esd_power_start": (i32, [vp, vp]),
            "esd_matrix_diag_scale": (i32, [vp, vp]),
            "esd_set_precision": (i32, [vp, i32, f64]),
            "esd_solver_set_precond_matrix": (i32, [vp, vp]),
            "esd_power_estimate": (i32, [vp, P(f64), P(i32), vp]),
            "esd_paper_cond_estimate": (i32, [vp, P(f64), P(f64), P(f64)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def esd_last_error() -> str:
    return lib().esd_last_error().decode()


def _check(code, allow=()):
    if code != OK and code not in allow:
        raise EsdError(code, esd_last_error())
    return code


def _ptr(a):
    """Device or host address of a torch tensor / NumPy array (contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not (a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]):
            raise ValueError("array must be contiguous")
        return C.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_ok(a, kind):
    if a is None:
        return
    if hasattr(a, "dtype") and hasattr(a, "data_ptr"):
        import torch
        want = {"f64": torch.float64, "i32": torch.int32}[kind]
        if a.dtype != want:
            raise TypeError(f"expected {want}, got {a.dtype}")
    elif isinstance(a, np.ndarray):
        want = {"f64": np.float64, "i32": np.int32}[kind]
        if a.dtype != want:
            raise TypeError(f"expected {want}, got {a.dtype}")


def current_stream():
    """torch's current CUDA stream handle when torch has CUDA, else 0 (legacy stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


# ---------------------------------------------------------------- C-named functions

def esd_create_matrix(n, nnz, rowptr, colind, val, colour_ptr, ncolours, flags=0, stream=None):
    _dtype_ok(rowptr, "i32"), _dtype_ok(colind, "i32"), _dtype_ok(val, "f64")
    cp = np.ascontiguousarray(colour_ptr, dtype=np.int32)
    out = C.c_void_p()
    st = current_stream() if stream is None else stream
    _check(lib().esd_create_matrix(n, nnz, _ptr(rowptr), _ptr(colind), _ptr(val), _ptr(cp), ncolours, flags,
                                   C.c_void_p(st), C.byref(out)))
    return out


def esd_matrix_destroy(h):
    return _check(lib().esd_matrix_destroy(h))


def esd_matrix_diag_scale(h, d):
    """d (n doubles, NumPy or CUDA tensor) receives 1/sqrt(a_ii) of a scaled matrix."""
    _check(lib().esd_matrix_diag_scale(h, _ptr(d)))


def esd_matrix_info(h):
    n, ncol, fl, bl = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    nnz = C.c_int64()
    _check(lib().esd_matrix_info(h, C.byref(n), C.byref(nnz), C.byref(ncol), C.byref(fl), C.byref(bl)))
    return dict(n=n.value, nnz=nnz.value, ncolours=ncol.value, fwd_levels=fl.value, bwd_levels=bl.value)


def esd_matrix_layout(h):
    """Which parts (A, L, U) have the column-free FP32 copy, the values each holds, and the
    number of 32-row slices."""
    cf = (C.c_int32 * 3)()
    ent = (C.c_int64 * 3)()
    ns = C.c_int32()
    _check(lib().esd_matrix_layout(h, cf, ent, C.byref(ns)))
    return dict(column_free=[bool(v) for v in cf], slot_entries=list(ent), slices=ns.value)


def esd_factor_ic0(h, max_tries=30):
    s = C.c_double()
    _check(lib().esd_factor_ic0(h, max_tries, C.byref(s)))
    return s.value


def esd_matrix_spmv(h, x, y):
    _check(lib().esd_matrix_spmv(h, _ptr(x), _ptr(y)))


def esd_matrix_apply_ic(h, r, z):
    _check(lib().esd_matrix_apply_ic(h, _ptr(r), _ptr(z)))


def esd_pattern_grad(h, lam, x, grad):
    _check(lib().esd_pattern_grad(h, _ptr(lam), _ptr(x), _ptr(grad)))


def esd_matrix_set_values(h, val):
    _dtype_ok(val, "f64")
    _check(lib().esd_matrix_set_values(h, _ptr(val)))


def esd_fv_assemble(h, grid: EsdFvGrid, theta, cell_row):
    _dtype_ok(theta, "f64"), _dtype_ok(cell_row, "i32")
    _check(lib().esd_fv_assemble(h, C.byref(grid), _ptr(theta), _ptr(cell_row)))


def esd_fv_grad_theta(h, grid: EsdFvGrid, theta, cell_row, lam, x, grad_theta):
    for a in (theta, lam, x, grad_theta):
        _dtype_ok(a, "f64")
    _dtype_ok(cell_row, "i32")
    _check(lib().esd_fv_grad_theta(h, C.byref(grid), _ptr(theta), _ptr(cell_row), _ptr(lam), _ptr(x),
                                   _ptr(grad_theta)))


def esd_refresh_W(h):
    _check(lib().esd_refresh_W(h))


def esd_params_default():
    p = EsdParams()
    lib().esd_params_default(C.byref(p))
    return p


def esd_solver_create(mh, params=None):
    out = C.c_void_p()
    p = params if params is not None else esd_params_default()
    _check(lib().esd_solver_create(mh, C.byref(p), C.byref(out)))
    return out


def esd_solver_destroy(h):
    return _check(lib().esd_solver_destroy(h))


def esd_set_mode(h, mode):
    _check(lib().esd_set_mode(h, mode))


def esd_solve(h, b, x, tol, maxit, sample_m=0):
    """Returns (status, iters, relres); status OK or ERR_MAXIT (other errors raise)."""
    it, rr = C.c_int32(), C.c_double()
    st = _check(lib().esd_solve(h, _ptr(b), _ptr(x), tol, maxit, sample_m, C.byref(it), C.byref(rr)),
                allow=(ERR_MAXIT,))
    return st, it.value, rr.value


def esd_solve_pair(h1, h2, b1, x1, b2, x2, tol, maxit):
    """Two systems with the same matrix together (both solvers in the refinement form, plain
    mode). Returns (status, (iters1, relres1), (iters2, relres2), paired): status OK or
    ERR_MAXIT (other errors raise), paired the iterations the paired kernels ran."""
    i1, r1, i2, r2, pr = C.c_int32(), C.c_double(), C.c_int32(), C.c_double(), C.c_int32()
    st = _check(lib().esd_solve_pair(h1, h2, _ptr(b1), _ptr(x1), _ptr(b2), _ptr(x2), tol, maxit, C.byref(i1),
                                     C.byref(r1), C.byref(i2), C.byref(r2), C.byref(pr)), allow=(ERR_MAXIT,))
    return st, (i1.value, r1.value), (i2.value, r2.value), pr.value


def esd_true_relres(h):
    v = C.c_double()
    _check(lib().esd_true_relres(h, C.byref(v)))
    return v.value


def esd_last_solve_info(h):
    """dict(iters, outer_steps, first_inner, restarts, max_gap, true_relres, status) of the
    last solve."""
    it, outer, first, rs, st = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    gap, rr = C.c_double(), C.c_double()
    _check(lib().esd_last_solve_info(h, C.byref(it), C.byref(outer), C.byref(first), C.byref(rs),
                                     C.byref(gap), C.byref(rr), C.byref(st)))
    return {"iters": it.value, "outer_steps": outer.value, "first_inner": first.value,
            "restarts": rs.value, "max_gap": gap.value, "true_relres": rr.value, "status": st.value}


def esd_sample_and_build_W(h, theta=math.inf):
    m = C.c_int32()
    _check(lib().esd_sample_and_build_W(h, theta, C.byref(m)))
    return m.value


def esd_set_W(h, W, m):
    _check(lib().esd_set_W(h, _ptr(W), m))


def esd_get_W(h, n, m_cap=64):
    """Returns (W, AW, E) as NumPy arrays (n x m column-major, n x m, m x m)."""
    m = C.c_int32()
    W = np.zeros((n, m_cap), order="F")
    AW = np.zeros((n, m_cap), order="F")
    E = np.zeros(m_cap * m_cap)
    _check(lib().esd_get_W(h, _ptr(W), _ptr(AW), _ptr(E), C.byref(m)))
    k = m.value
    return W[:, :k].copy(order="F"), AW[:, :k].copy(order="F"), E[: k * k].reshape(k, k)


def esd_ritz_values(h, cap=64):
    out = np.zeros(cap)
    cnt = C.c_int32()
    _check(lib().esd_ritz_values(h, _ptr(out), cap, C.byref(cnt)))
    return out[: min(cnt.value, cap)]


def esd_estimate_cond(h):
    lo, hi, k, r = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    _check(lib().esd_estimate_cond(h, C.byref(lo), C.byref(hi), C.byref(k), C.byref(r)))
    return lo.value, hi.value, k.value, r.value


def esd_solver_set_precond_matrix(h, P):
    _check(lib().esd_solver_set_precond_matrix(h, P))


def esd_set_precision(h, precision, inner_tol=0.1):
    _check(lib().esd_set_precision(h, precision, inner_tol))


def esd_power_start(h, v0):
    """v0: n doubles (NumPy or CUDA tensor), or None to stop the power method."""
    _check(lib().esd_power_start(h, None if v0 is None else _ptr(v0)))


def esd_power_estimate(h, v=None):
    """(lambda_max, steps); v (n doubles, optional) receives the unit power vector."""
    lam, k = C.c_double(), C.c_int32()
    _check(lib().esd_power_estimate(h, C.byref(lam), C.byref(k), None if v is None else _ptr(v)))
    return lam.value, k.value


def esd_paper_cond_estimate(h):
    """(lambda_max, lambda_min, kappa) of Algorithm PCG-con, formed by the library."""
    lmax, lmin, kap = C.c_double(), C.c_double(), C.c_double()
    _check(lib().esd_paper_cond_estimate(h, C.byref(lmax), C.byref(lmin), C.byref(kap)))
    return lmax.value, lmin.value, kap.value


def esd_get_history(h, cap):
    a, b = np.zeros(cap), np.zeros(cap)
    cnt = C.c_int32()
    _check(lib().esd_get_history(h, _ptr(a), _ptr(b), cap, C.byref(cnt)))
    k = min(cnt.value, cap)
    return a[:k], b[: max(k - 1, 0)]


def esd_get_samples(h, n, cap):
    s = np.zeros((n, cap), order="F")
    it = np.zeros(cap, dtype=np.int32)
    m = C.c_int32()
    _check(lib().esd_get_samples(h, _ptr(s), _ptr(it), cap, C.byref(m)))
    k = min(m.value, cap)
    return s[:, :k], it[:k]


def esd_backward_euler_rhs(h, x_prev, s, inv_dt, b):
    _check(lib().esd_backward_euler_rhs(h, _ptr(x_prev), _ptr(s), inv_dt, _ptr(b)))


def esd_profile_iterations(h, b, x, reps, cap=64):
    """Returns [(kernel name, average ms per launch)] for one iteration of the current mode."""
    ms = np.zeros(cap)
    names = C.create_string_buffer(32 * cap)
    cnt = C.c_int32()
    _check(lib().esd_profile_iterations(h, _ptr(b), _ptr(x), reps, _ptr(ms), names, cap, C.byref(cnt)))
    k = min(cnt.value, cap)
    raw = names.raw
    return [(raw[32 * j: 32 * j + 32].split(b"\0")[0].decode(), float(ms[j])) for j in range(k)]


def esd_profile_pair_iterations(h1, h2, b1, x1, b2, x2, reps, cap=64):
    """[(kernel name, average ms per launch)] for one paired iteration of two systems."""
    ms = np.zeros(cap)
    names = C.create_string_buffer(32 * cap)
    cnt = C.c_int32()
    _check(lib().esd_profile_pair_iterations(h1, h2, _ptr(b1), _ptr(x1), _ptr(b2), _ptr(x2), reps, _ptr(ms), names,
                                             cap, C.byref(cnt)))
    k = min(cnt.value, cap)
    raw = names.raw
    return [(raw[32 * j: 32 * j + 32].split(b"\0")[0].decode(), float(ms[j])) for j in range(k)]


def esd_lanczos_extremes_noalloc(alpha, beta, k, out, stream=None):
    """Condition estimate from caller-owned device arrays, allocating nothing (for callers
    that cannot call cudaMalloc). alpha: k doubles, beta: k-1 doubles (may be None when
    k = 1), out: 3 doubles (lmin, lmax, kappa); all contiguous CUDA float64 tensors."""
    import torch
    for name, t, need in (("alpha", alpha, k), ("beta", beta, k - 1), ("out", out, 3)):
        if t is None and need <= 0:
            continue
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} values, {need} needed")
    st = current_stream() if stream is None else stream
    _check(lib().esd_lanczos_extremes_noalloc(_ptr(alpha), _ptr(beta), k, _ptr(out), C.c_void_p(st)))


# ---------------------------------------------------------------- handle owners

class Matrix:
    """Library copy of an SPD CSR matrix in colour-major order (``esd_create_matrix``)."""

    def __init__(self, rowptr, colind, val, colour_ptr, stream=None, diag_scale=False):
        n = len(rowptr) - 1
        nnz = len(colind)
        self.n, self.nnz = n, nnz
        flags = MATRIX_DIAG_SCALE if diag_scale else 0
        self._h = esd_create_matrix(n, nnz, rowptr, colind, val, colour_ptr, len(colour_ptr) - 1, flags, stream)
        self.shift = None

    @classmethod
    def from_problem(cls, prob, stream=None, diag_scale=False):
        return cls(np.ascontiguousarray(prob.rowptr, np.int32), np.ascontiguousarray(prob.colind, np.int32),
                   np.ascontiguousarray(prob.val, np.float64), prob.colour_ptr, stream, diag_scale)

    def diag_scale(self):
        """d = 1/sqrt(diag(A)) of a matrix created with diag_scale=True (the library holds
        D^-1/2 A D^-1/2: solve with b^ = d b, then x = d x^)."""
        d = np.zeros(self.n)
        esd_matrix_diag_scale(self._h, d)
        return d

    @property
    def handle(self):
        return self._h

    def info(self):
        return esd_matrix_info(self._h)

    def layout(self):
        return esd_matrix_layout(self._h)

    def factor_ic0(self, max_tries=30):
        self.shift = esd_factor_ic0(self._h, max_tries)
        return self.shift

    def spmv(self, x, y):
        esd_matrix_spmv(self._h, x, y)

    def apply_ic(self, r, z):
        esd_matrix_apply_ic(self._h, r, z)

    def pattern_grad(self, lam, x, grad):
        esd_pattern_grad(self._h, lam, x, grad)

    def set_values(self, val):
        esd_matrix_set_values(self._h, val)

    def close(self):
        if getattr(self, "_h", None):
            esd_matrix_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """``esd_solver`` bound to a Matrix; keeps the matrix alive."""

    def __init__(self, matrix: Matrix, precond=PRECOND_IC0, maxit_cap=20000, sample_cap=32, lmax=0,
                 rank_tol=1e-12, precision=FP64, inner_tol=0.1, max_outer=60, resume_direction=1,
                 sampling=SAMPLING_A):
        p = esd_params_default()
        p.precond, p.maxit_cap, p.sample_cap, p.lmax = precond, maxit_cap, sample_cap, lmax
        p.rank_tol, p.precision, p.inner_tol, p.max_outer = rank_tol, precision, inner_tol, max_outer
        p.resume_direction = resume_direction
        p.sampling = sampling
        self.matrix = matrix
        self.maxit_cap = maxit_cap
        self._h = esd_solver_create(matrix.handle, p)

    def set_mode(self, mode):
        esd_set_mode(self._h, mode)

    def set_precision(self, precision, inner_tol=0.1):
        esd_set_precision(self._h, precision, inner_tol)

    def set_precond_matrix(self, P):
        """Precondition with IC(0) of another Matrix P (same rows and colours as A), e.g. the
        block-diagonal part of A for block-Jacobi IC; None returns to A's own factor."""
        esd_solver_set_precond_matrix(self._h, None if P is None else P.handle)
        self._precond_matrix = P  # keep it alive while the solver uses it

    def solve(self, b, x, tol=1e-8, maxit=None, sample_m=0):
        return esd_solve(self._h, b, x, tol, maxit or self.maxit_cap, sample_m)

    def solve_pair(self, other, b1, x1, b2, x2, tol=1e-8, maxit=None):
        """This solver's system and `other`'s solved together (esd_solve_pair)."""
        return esd_solve_pair(self._h, other._h, b1, x1, b2, x2, tol, maxit or min(self.maxit_cap, other.maxit_cap))

    def true_relres(self):
        return esd_true_relres(self._h)

    def last_solve_info(self):
        return esd_last_solve_info(self._h)

    def sample_and_build_W(self, theta=math.inf):
        return esd_sample_and_build_W(self._h, theta)

    def set_W(self, W):
        W = np.asfortranarray(W, dtype=np.float64) if isinstance(W, np.ndarray) else W
        esd_set_W(self._h, W, W.shape[1])

    def get_W(self):
        return esd_get_W(self._h, self.matrix.n)

    def refresh_W(self):
        esd_refresh_W(self._h)

    def ritz_values(self):
        return esd_ritz_values(self._h)

    def estimate_cond(self):
        return esd_estimate_cond(self._h)

    def power_start(self, v0):
        """Start (or, with None, stop) the power method of Algorithm PCG-con (Section 5.4)."""
        v0 = np.ascontiguousarray(v0, dtype=np.float64) if isinstance(v0, np.ndarray) else v0
        esd_power_start(self._h, v0)

    def power_estimate(self, vector=False):
        """(lambda_max, steps) of the power method, plus the unit vector when asked."""
        if not vector:
            return esd_power_estimate(self._h)
        v = np.zeros(self.matrix.n)
        lam, k = esd_power_estimate(self._h, v)
        return lam, k, v

    def paper_cond_estimate(self):
        """Algorithm PCG-con's kappa = lambda_max / lambda_min: lambda_max from the power
        method, lambda_min the smallest Ritz value of the current W (after
        sample_and_build_W with theta = inf on the sampled solve). Returns (lmax, lmin, kappa)."""
        return esd_paper_cond_estimate(self._h)

    def history(self):
        return esd_get_history(self._h, self.maxit_cap)

    def samples(self, cap=64):
        return esd_get_samples(self._h, self.matrix.n, cap)

    def profile_iterations(self, b, x, reps=20):
        return esd_profile_iterations(self._h, b, x, reps)

    def profile_pair_iterations(self, other, b1, x1, b2, x2, reps=20):
        return esd_profile_pair_iterations(self._h, other._h, b1, x1, b2, x2, reps)

    def backward_euler_rhs(self, x_prev, s, inv_dt, b):
        esd_backward_euler_rhs(self._h, x_prev, s, inv_dt, b)

    def close(self):
        if getattr(self, "_h", None):
            esd_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

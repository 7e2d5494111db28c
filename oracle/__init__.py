"""CPU oracle (FP64) for error-vector-sampling deflation and subspace correction ICCG.

TEST INFRASTRUCTURE ONLY. It is imported by ``tests/``, by the package smoke check and by
the benchmark's CPU-baseline leg; the library's product path never touches it. It shares
no code with the CUDA path: the Krylov iterations, IC(0), the substitutions and the power
method are plain C loops (``esd_oracle.c``); the auxiliary-matrix construction, the Lanczos
estimate, the diagonal scaling and the adjoint chain rule are plain NumPy/SciPy (library
primitives as single steps: ``eigh``, ``cholesky``, sparse matvec, tridiagonal
eigenvalues). Any IC(0) factor can precondition a ``System``, so block-Jacobi IC is
``System(A, IC0(block-diagonal part of A))``.

Every function cites the passage of arXiv 2203.08498 it follows. Where the paper is silent
the reading is stated in the docstring.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "esd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libesd_oracle.so")
_OMP_PATH = os.path.join(_HERE, "_build", "libesd_oracle_omp.so")
_lib = None
_lock = threading.Lock()

OK, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_MAXIT, ERR_STATE = 0, -2, -3, -4, -5
PLAIN, DEFLATION, SUBSPACE_CORRECTION = 0, 1, 2


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build``: -O2 with floating-point contraction off,
    so every product is rounded before it is added and x86 and Arm builds agree bit for bit.
    ``openmp`` builds the all-core variant of the same source (identical results)."""
    path = _OMP_PATH if openmp else _LIB_PATH
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".{os.getpid()}.tmp"
        extra = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", *extra, "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


class _System(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("rp", C.c_void_p), ("ci", C.c_void_p), ("va", C.c_void_p),
        ("ncol", C.c_int), ("cp", C.c_void_p), ("precond", C.c_int),
        ("Lrp", C.c_void_p), ("Lci", C.c_void_p), ("Lva", C.c_void_p),
        ("Urp", C.c_void_p), ("Uj", C.c_void_p), ("Ua", C.c_void_p),
        ("mode", C.c_int), ("m", C.c_int), ("W", C.c_void_p), ("AW", C.c_void_p),
        ("LE", C.c_void_p),
    ]


class _SolveIO(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("maxit", C.c_int), ("sample_m", C.c_int), ("lmax", C.c_int),
        ("sample_method", C.c_int),
        ("samples", C.c_void_p), ("sample_iter", C.c_void_p), ("alpha_hist", C.c_void_p),
        ("beta_hist", C.c_void_p), ("res_hist", C.c_void_p), ("wtr_hist", C.c_void_p),
        ("iters", C.c_int), ("relres", C.c_double), ("status", C.c_int),
    ]


def load(path: str):
    """Load a compiled oracle library and declare its signatures."""
    L = C.CDLL(path)
    vp, i32, f64 = C.c_void_p, C.c_int, C.c_double
    L.orc_dot.restype = f64
    L.orc_dot.argtypes = [C.c_long, vp, vp]
    L.orc_spmv.argtypes = [i32, vp, vp, vp, vp, vp]
    L.orc_ic0.restype = i32
    L.orc_ic0.argtypes = [i32, vp, vp, vp, i32, vp, vp, vp, C.POINTER(f64)]
    L.orc_tril_nnz.restype = C.c_long
    L.orc_tril_nnz.argtypes = [i32, vp, vp]
    L.orc_ic_apply.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.orc_ic_transpose.restype = C.c_long
    L.orc_ic_transpose.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp]
    L.orc_precond.argtypes = [C.POINTER(_System), vp, vp, vp]
    L.orc_solve.restype = i32
    L.orc_solve.argtypes = [C.POINTER(_System), vp, vp, C.POINTER(_SolveIO)]
    L.orc_sampling_a_schedule.argtypes = [i32, i32, i32, vp]
    L.orc_threads.restype = i32
    L.orc_threads.argtypes = []
    L.orc_power_method.restype = f64
    L.orc_power_method.argtypes = [i32, vp, vp, vp, vp, i32, vp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


class using:
    """``with oracle.using(openmp_lib()):`` routes every oracle call to that library."""

    def __init__(self, library):
        self.library = library

    def __enter__(self):
        global _lib
        self.saved, _lib = lib(), self.library
        return self.library

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def openmp_lib():
    """The OpenMP build of the same oracle (bit-identical results), for timing on all host
    cores; OMP_NUM_THREADS sets its threads."""
    return load(build(openmp=True))


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ------------------------------------------------------------------ kernels

def dot(x, y) -> float:
    """Pairwise-summed FP64 dot product."""
    x, y = _c(x, np.float64), _c(y, np.float64)
    return lib().orc_dot(len(x), _p(x), _p(y))


def spmv(prob, x):
    x = _c(x, np.float64)
    y = np.empty(prob.n)
    lib().orc_spmv(prob.n, _p(prob.rowptr), _p(prob.colind), _p(prob.val), _p(x), _p(y))
    return y


def diag_scale(prob):
    """Symmetric Jacobi scaling of the test matrices (Sections 5.1, 5.4): ``A^ = D^-1/2 A
    D^-1/2`` with ``D = diag(A)``, entry by entry ``a^_ij = (a_ij d_i) d_j`` for
    ``d_i = 1/sqrt(a_ii)``. Returns (a copy of the problem holding A^, d). A solve of
    ``A x = b`` is the solve of ``A^ x^ = d * b`` with ``x = d * x^``."""
    import copy
    rp = np.asarray(prob.rowptr, dtype=np.int64)
    ci = np.asarray(prob.colind, dtype=np.int64)
    va = np.asarray(prob.val, dtype=np.float64)
    rows = np.repeat(np.arange(prob.n), np.diff(rp))
    diag = va[rows == ci]
    if len(diag) != prob.n or not np.all(diag > 0) or not np.all(np.isfinite(diag)):
        raise ValueError("diagonal scaling needs a positive finite diagonal entry in every row")
    d = 1.0 / np.sqrt(diag)
    out = copy.copy(prob)
    out.val = (va * d[rows]) * d[ci]
    return out, d


class IC0:
    """IC(0) factor ``M = L L^T``, ``L`` on the pattern of tril(A) (diagonal last per row).

    The paper uses incomplete Cholesky preconditioning without stating the fill level
    (Section 4.4 treats its cost as that of one SpMV, which implies zero fill). Reading:
    IC(0) in the multicolour order fixed by the problem; if a pivot is not positive the
    factorisation is retried on ``A + a diag(A)`` with ``a = 1e-3, 2e-3, 4e-3, ...``.
    """

    def __init__(self, prob, max_tries: int = 30):
        self.n = prob.n
        rp, ci, va = _c(prob.rowptr, np.int32), _c(prob.colind, np.int32), _c(prob.val, np.float64)
        nl = lib().orc_tril_nnz(prob.n, _p(rp), _p(ci))
        self.Lrp = np.zeros(prob.n + 1, dtype=np.int32)
        self.Lci = np.zeros(nl, dtype=np.int32)
        self.Lva = np.zeros(nl, dtype=np.float64)
        sh = C.c_double(0.0)
        st = lib().orc_ic0(prob.n, _p(rp), _p(ci), _p(va), max_tries, _p(self.Lrp), _p(self.Lci),
                           _p(self.Lva), C.byref(sh))
        if st != OK:
            raise ArithmeticError("IC(0) breakdown: matrix not SPD enough for the shift rule")
        self.shift = sh.value
        self.colour_ptr = _c(prob.colour_ptr, np.int32)
        # column index of L for the backward sweep (later colours first, rows ascending)
        self.Urp = np.zeros(prob.n + 1, dtype=np.int32)
        self.Uj = np.zeros(max(nl - prob.n, 1), dtype=np.int32)
        self.Ua = np.zeros(max(nl - prob.n, 1), dtype=np.int32)
        lib().orc_ic_transpose(prob.n, len(self.colour_ptr) - 1, _p(self.colour_ptr), _p(self.Lrp), _p(self.Lci),
                               _p(self.Urp), _p(self.Uj), _p(self.Ua))

    def dense_L(self):
        return sp.csr_matrix((self.Lva, self.Lci, self.Lrp), shape=(self.n, self.n)).toarray()

    def apply(self, r):
        """``z = (L L^T)^{-1} r`` by colour-ordered forward and backward substitution."""
        r = _c(r, np.float64)
        z = np.empty(self.n)
        y = np.empty(self.n)
        lib().orc_ic_apply(self.n, len(self.colour_ptr) - 1, _p(self.colour_ptr), _p(self.Lrp),
                           _p(self.Lci), _p(self.Lva), _p(self.Urp), _p(self.Uj), _p(self.Ua), _p(r), _p(z), _p(y))
        return z


# ------------------------------------------------------------------ auxiliary matrix

class Aux:
    """W, AW = A W, E = W^T A W and its Cholesky factor (Eq. mc, Eq. deflation:projector)."""

    def __init__(self, W, AW, E):
        self.W = np.asfortranarray(W, dtype=np.float64)
        self.AW = np.asfortranarray(AW, dtype=np.float64)
        self.E = np.asarray(E, dtype=np.float64)
        self.m = self.W.shape[1]
        self.LE = np.ascontiguousarray(np.linalg.cholesky(self.E))
        self.ritz = np.linalg.eigvalsh(self.E)

    @classmethod
    def from_basis(cls, prob, W):
        W = np.asarray(W, dtype=np.float64)
        AW = prob.scipy() @ W
        E = W.T @ AW
        return cls(W, AW, 0.5 * (E + E.T))


def mgs(X, passes: int = 2):
    """Modified Gram-Schmidt with one re-orthogonalisation pass (Eq. ekd)."""
    X = np.array(X, dtype=np.float64, copy=True)
    m = X.shape[1]
    for j in range(m):
        for _ in range(passes):
            for k in range(j):
                X[:, j] -= (X[:, k] @ X[:, j]) * X[:, k]
        X[:, j] /= np.linalg.norm(X[:, j])
    return X


def build_w(prob, x, samples, sample_iter, rank_tol: float = 1e-12, theta: float = np.inf):
    """Auxiliary matrix from sampled iterates (Section 4.2, Eq. ek, ekd, Rayleigh-Ritz, bk).

    1. ``e_s = x - x~_s`` for every filled slot (Eq. ek);
    2. columns normalised; ``G = Ehat^T Ehat``; the rank ``mbar`` counts the eigenvalues of
       G above ``rank_tol * max eig`` (reading: the paper gives no tolerance);
    3. an orthonormal basis by modified Gram-Schmidt (Eq. ekd) of ``Ehat`` when full rank,
       else of ``Ehat V_k`` (the kept eigen-directions of G, same span);
    4. ``theta = inf`` (default) keeps the whole basis, ``W = Q``; a finite theta keeps the
       Ritz vectors ``Q t_i`` of ``Q^T A Q t = lambda t`` with ``lambda < theta`` (Eq. bk);
    5. ``AW = A W``, ``E = W^T A W``, ``chol(E)``.
    Returns (Aux, info dict).
    """
    filled = [k for k in range(samples.shape[1]) if sample_iter[k] > 0]
    Eh = x[:, None] - samples[:, filled]
    nrm = np.linalg.norm(Eh, axis=0)
    keepc = nrm > 0
    Eh = Eh[:, keepc] / nrm[keepc]
    G = Eh.T @ Eh
    ev, V = np.linalg.eigh(G)
    keep = ev > rank_tol * ev.max()
    basis = Eh if keep.all() else Eh @ V[:, keep]
    Q = mgs(basis)
    A = prob.scipy()
    AQ = A @ Q
    EQ = Q.T @ AQ
    EQ = 0.5 * (EQ + EQ.T)
    ritz, T = np.linalg.eigh(EQ)
    if np.isfinite(theta):
        sel = ritz < theta
        W, AW = Q @ T[:, sel], AQ @ T[:, sel]
        E = np.diag(ritz[sel])
    else:
        W, AW, E = Q, AQ, EQ
    info = dict(m_filled=len(filled), mbar=int(keep.sum()), ritz=ritz, m_kept=W.shape[1])
    return Aux(W, AW, E), info


# ------------------------------------------------------------------ solver

def default_lmax(m: int, maxit: int) -> int:
    """Smallest l with m^l > N_max (Appendix A)."""
    l, p = 0, 1
    while p <= maxit:
        p *= m
        l += 1
    return l


def sampling_a_schedule(m: int, N: int, lmax: int | None = None):
    """Per slot, the iteration whose iterate method A keeps when the solve stops at N."""
    lmax = default_lmax(m, max(N, 1)) if lmax is None else lmax
    out = np.zeros(m, dtype=np.int32)
    lib().orc_sampling_a_schedule(m, lmax, N, _p(out))
    return out


class System:
    """A (CSR), optional IC(0) factor and optional auxiliary matrix, in one of the modes."""

    def __init__(self, prob, ic: IC0 | None, mode: int = PLAIN, aux: Aux | None = None):
        if mode != PLAIN and aux is None:
            raise ValueError("deflation / subspace correction need W")
        if aux is not None and aux.m > 64:
            raise ValueError("the oracle supports m <= 64")
        self.prob, self.ic, self.mode, self.aux = prob, ic, mode, aux
        self._keep = [_c(prob.rowptr, np.int32), _c(prob.colind, np.int32), _c(prob.val, np.float64),
                      _c(prob.colour_ptr, np.int32)]
        rp, ci, va, cp = self._keep
        s = _System()
        s.n, s.rp, s.ci, s.va = prob.n, _p(rp), _p(ci), _p(va)
        s.ncol, s.cp = len(cp) - 1, _p(cp)
        s.precond = 1 if ic is not None else 0
        if ic is not None:
            s.Lrp, s.Lci, s.Lva = _p(ic.Lrp), _p(ic.Lci), _p(ic.Lva)
            s.Urp, s.Uj, s.Ua = _p(ic.Urp), _p(ic.Uj), _p(ic.Ua)
        s.mode = mode
        if aux is not None:
            s.m, s.W, s.AW, s.LE = aux.m, _p(aux.W), _p(aux.AW), _p(aux.LE)
        self._s = s

    def precond(self, r):
        """``z = M^{-1} r`` (+ ``W E^{-1} W^T r`` in subspace-correction mode, Eq. mc)."""
        r = _c(r, np.float64)
        z = np.empty_like(r)
        w = np.empty_like(r)
        lib().orc_precond(C.byref(self._s), _p(r), _p(z), _p(w))
        return z

    def solve(self, b, x0=None, tol: float = 1e-8, maxit: int = 20000, sample_m: int = 0,
              lmax: int | None = None, history: bool = True, sample_method: int = 0):
        """PCG / deflated PCG (Algorithm PCG-con without the power method; Algorithm DPCG).

        Stops when ``||r_i||_2 <= tol ||b||_2``; the iteration count is the number of
        alpha steps. ``sample_m > 0`` stores iterates by sampling method A (Appendix A;
        ``sample_method = 0``) or B (Section 4.2, ``sample_method = 1``: the iterate whose
        relative residual first reaches ``tol^(s/(m+1))``, s = 1..m; an iteration that first
        reaches several levels is stored once; slots are filled in order).
        """
        n = self.prob.n
        b = _c(b, np.float64)
        x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        io = _SolveIO()
        io.tol, io.maxit, io.sample_m, io.sample_method = tol, maxit, sample_m, sample_method
        io.lmax = default_lmax(sample_m, maxit) if (sample_m > 1 and lmax is None) else (lmax or 0)
        samples = np.zeros((n, sample_m), order="F") if sample_m > 0 else None
        siter = np.zeros(max(sample_m, 1), dtype=np.int32)
        ah = np.zeros(maxit) if history else None
        bh = np.zeros(maxit) if history else None
        rh = np.zeros(maxit + 1) if history else None
        wh = np.zeros(maxit + 1) if history else None
        io.samples, io.sample_iter = _p(samples), _p(siter)
        io.alpha_hist, io.beta_hist, io.res_hist, io.wtr_hist = _p(ah), _p(bh), _p(rh), _p(wh)
        lib().orc_solve(C.byref(self._s), _p(b), _p(x), C.byref(io))
        k = io.iters
        out = dict(x=x, iters=k, relres=io.relres, status=io.status, samples=samples,
                   sample_iter=siter[:sample_m] if sample_m else siter[:0])
        if history:
            out.update(alpha=ah[:k], beta=bh[:max(k - 1, 0)], res=rh[:k + 1], wtr=wh[:k + 1])
        return out


def lanczos_tridiagonal(alpha, beta):
    """Lanczos matrix of the CG run from its coefficients (Saad, Iterative Methods, 6.7.3):
    ``T_jj = 1/a_j + b_{j-1}/a_{j-1}`` (the second term absent for j = 0) and
    ``T_{j,j+1} = sqrt(b_j)/a_j``. Here ``b_j`` is the coefficient in ``p_{j+1} = z_{j+1} +
    b_j p_j``. Returns the diagonal and the off-diagonal."""
    a = np.asarray(alpha, dtype=np.float64)
    b = np.asarray(beta, dtype=np.float64)[: len(a) - 1]
    d = 1.0 / a
    d[1:] += b / a[:-1]
    e = np.sqrt(b) / a[:-1]
    return d, e


def estimate_cond(alpha, beta):
    """Extreme eigenvalues of the CG Lanczos matrix and their ratio (SciPy's tridiagonal
    eigensolver as the library step)."""
    d, e = lanczos_tridiagonal(alpha, beta)
    if len(d) == 0:
        return np.nan, np.nan, np.nan
    ev = sla.eigvalsh_tridiagonal(d, e) if len(d) > 1 else d
    return float(ev.min()), float(ev.max()), float(ev.max() / ev.min())


def power_method(prob, v0, k: int):
    """Power method of Algorithm PCG-con (Section 5.4) on A: ``v_0 = v0/||v0||``, then
    ``v_i = A v_{i-1} / ||A v_{i-1}||`` for i = 1..k, and ``lambda_max = (v_k, A v_k)``.
    In the algorithm each CG iteration takes one step (its SpMV multiplies ``(p_i, v_{i-1})``
    together); the vectors do not depend on the CG iterates, so k steps here equal a
    k-iteration solve. Returns (lambda_max, v_k); NaN when a norm vanishes."""
    v = np.array(v0, dtype=np.float64, copy=True)
    w = np.empty(prob.n)
    rp, ci, va = _c(prob.rowptr, np.int32), _c(prob.colind, np.int32), _c(prob.val, np.float64)
    lam = lib().orc_power_method(prob.n, _p(rp), _p(ci), _p(va), _p(v), int(k), _p(w))
    return float(lam), v


def pcg_cond_estimate(prob, b, v0, m: int, tol: float = 1e-8, maxit: int = 20000, precond: bool = True):
    """Algorithm PCG-con (Section 5.4): PCG on ``A x = b`` (IC(0), or none with
    ``precond=False``) with m iterates sampled (method A), the power method for
    ``lambda_max`` (one step per iteration), the sampled errors made orthonormal (Eq. ek,
    ekd) and the smallest Ritz value of ``E^T A E`` (Eq. Rayleigh-Ritz) for ``lambda_min``;
    ``kappa = lambda_max / lambda_min``."""
    sysm = System(prob, IC0(prob) if precond else None)
    out = sysm.solve(b, tol=tol, maxit=maxit, sample_m=m, history=False)
    lam_max, v = power_method(prob, v0, out["iters"])
    aux, info = build_w(prob, out["x"], out["samples"], out["sample_iter"])
    lam_min = float(info["ritz"][0])
    return dict(x=out["x"], iters=out["iters"], lmax=lam_max, lmin=lam_min, kappa=lam_max / lam_min, v=v,
                ritz=info["ritz"])


# ------------------------------------------------------------------ sequence driver

def run_sequence(prob, T: int, mode: int, m: int, tol: float = 1e-8, maxit: int = 20000,
                 precond: bool = True, rhs=None):
    """Solve the sequence ``A x_t = b_t``, t = 1..T (Eq. ak2/ak3).

    System 1 is solved by plain ICCG while sampling method A stores ``m`` iterates; W is
    built from them (``build_w``) and reused for systems 2..T in ``mode``. The initial
    guess of system t is ``x_{t-1}`` (``x_0 = 0``). ``rhs(t, x_prev)`` gives ``b_t``; by
    default ``b_t = x_{t-1}/dt + s``.
    """
    ic = IC0(prob) if precond else None
    if rhs is None:
        def rhs(t, xp):
            return xp / prob.dt + prob.source
    x = np.zeros(prob.n)
    res = []
    aux = None
    for t in range(1, T + 1):
        b = rhs(t, x)
        if t == 1 or mode == PLAIN:
            sysm = System(prob, ic, PLAIN)
            out = sysm.solve(b, x, tol=tol, maxit=maxit, sample_m=(m if t == 1 and mode != PLAIN else 0))
            if t == 1 and mode != PLAIN:
                aux, info = build_w(prob, out["x"], out["samples"], out["sample_iter"])
        else:
            out = System(prob, ic, mode, aux).solve(b, x, tol=tol, maxit=maxit)
        x = out["x"]
        res.append(dict(iters=out["iters"], relres=out["relres"], status=out["status"], x=x.copy(),
                        alpha=out["alpha"], beta=out["beta"]))
    return res, aux


# ------------------------------------------------------------------ adjoint gradient
#
# Not part of the paper's method: the differentiation form built on it. For A(theta) x = b
# and a loss L(x), the adjoint lambda solves A^T lambda = dL/dx (A is symmetric, so this is
# one more system with the same matrix: it can reuse W and E); then dL/db = lambda and
# dL/da_ij = -lambda_i x_j on the pattern. The functions below carry that through the
# finite-volume assembly of the workloads (harmonic-mean faces, Dirichlet boundaries,
# k = exp(theta)) by the chain rule, face by face.

def _face_dT_dka(ka, kb, inv_h2):
    """d/dk_a of T = 2 k_a k_b / (k_a + k_b) / h^2."""
    return 2.0 * kb * kb / ((ka + kb) * (ka + kb)) * inv_h2


def _face_dL_dT(lam_a, lam_b, x_a, x_b):
    """dL/dT of one interior face: the sum of -lambda_i x_j over its four entries
    (+T at (a,a) and (b,b), -T at (a,b) and (b,a))."""
    return -(lam_a - lam_b) * (x_a - x_b)


def _boundary_dL_dk(lam_c, x_c, inv_h2):
    """A Dirichlet face adds 2 k_c / h^2 at (c, c): dL/dk_c = -lambda_c x_c 2 / h^2."""
    return -lam_c * x_c * 2.0 * inv_h2


def fv_theta_gradient(theta, h: float, lam, x):
    """dL/dtheta for the cell-centred FV operator A = I/dt + K(exp(theta)).

    ``theta``, ``lam`` and ``x`` are arrays of the grid's shape (axis 0 = x); the I/dt term
    does not depend on theta. Returns an array of the same shape.
    """
    theta = np.asarray(theta, dtype=np.float64)
    k = np.exp(theta)
    inv_h2 = 1.0 / (h * h)
    g = np.zeros_like(k)
    for ax in range(k.ndim):
        n_ax = k.shape[ax]
        lo = [slice(None)] * k.ndim
        hi = [slice(None)] * k.ndim
        lo[ax] = slice(0, n_ax - 1)
        hi[ax] = slice(1, n_ax)
        lo, hi = tuple(lo), tuple(hi)
        dLdT = _face_dL_dT(lam[lo], lam[hi], x[lo], x[hi])
        g[lo] += dLdT * _face_dT_dka(k[lo], k[hi], inv_h2)
        g[hi] += dLdT * _face_dT_dka(k[hi], k[lo], inv_h2)
        first = [slice(None)] * k.ndim
        last = [slice(None)] * k.ndim
        first[ax] = slice(0, 1)
        last[ax] = slice(n_ax - 1, n_ax)
        first, last = tuple(first), tuple(last)
        g[first] += _boundary_dL_dk(lam[first], x[first], inv_h2)
        g[last] += _boundary_dL_dk(lam[last], x[last], inv_h2)
    return k * g


def to_grid(prob, v):
    """Matrix-ordered vector -> array of the grid's shape (natural order, axis 0 = x)."""
    nat = np.empty(prob.n)
    nat[prob.perm] = v
    return nat.reshape(prob.shape, order="F")


def from_grid(prob, a):
    """Array of the grid's shape -> matrix-ordered vector."""
    return np.asarray(a).ravel(order="F")[prob.perm]


def adjoint_gradient(prob, theta, b, x_target, tol: float = 1e-13, maxit: int = 20000, mode: int = PLAIN,
                     aux: "Aux | None" = None):
    """Loss L = ||x - x_target||^2 with A(theta) x = b: forward ICCG, adjoint ICCG on
    A lambda = 2 (x - x_target) (same mode and auxiliary matrix), then dL/db = lambda and
    dL/dtheta by ``fv_theta_gradient``. ``prob`` is A(theta) with its ordering; vectors
    are in matrix order, theta and the returned grad_theta in grid shape."""
    ic = IC0(prob)
    sysm = System(prob, ic, mode, aux)
    x = sysm.solve(b, tol=tol, maxit=maxit, history=False)["x"]
    g = 2.0 * (x - x_target)
    lam = sysm.solve(g, tol=tol, maxit=maxit, history=False)["x"]
    grad_theta = fv_theta_gradient(theta, prob.h, to_grid(prob, lam), to_grid(prob, x))
    return {"x": x, "lambda": lam, "grad_b": lam, "grad_theta": grad_theta,
            "loss": float(np.dot(x - x_target, x - x_target))}

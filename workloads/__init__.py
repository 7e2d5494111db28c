"""Seeded synthetic workloads: the linear systems the solver and the oracle both consume.

This module defines *problems*, not the method: it assembles the SPD matrix of a
backward-Euler diffusion step (the sequence ``A x_t = b_t`` of Eq. ak2/ak3 with a fixed
``A``), its multicolour ordering, the source vectors and the seeded coefficient fields.
It holds none of the solver arithmetic (no CG, no preconditioner, no deflation); both the
CUDA path and the CPU oracle import it, and neither imports the other.

Readings of the workload descriptions (the paper is silent on them, it used SuiteSparse
matrices, Section 5.1):

* domain ``[0,1]^d`` with ``N`` cells per side, ``h = 1/N``, cell-centred finite volumes;
* ``A = I/dt + K`` with ``(K x)_i = sum_faces T_f (x_i - x_j)``, ``T_f`` the harmonic mean
  ``2 k_a k_b / (k_a + k_b) / h^2``; a Dirichlet (zero) boundary face adds ``2 k_i / h^2``;
* the right-hand side of system ``t`` is ``b_t = x_{t-1} / dt + s`` with ``x_0 = 0``;
* inclusions are placed by rejection sampling (no overlap, fully inside the domain);
* the ordering is colour-major: all rows of colour 0, then colour 1, ...; inside a colour
  the natural lexicographic order is kept. Colours are red-black ``(i+j) % 2`` in 2D and
  ``(i%2) + 2(j%2) + 4(k%2)`` in 3D.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Problem", "fv_diffusion", "square_inclusions", "sphere_inclusions",
    "gaussian_source", "smooth_gaussian_field", "config_c1", "config_c2", "config_c4",
    "small_3d", "random_spd_dense", "laplacian_1d", "ic0_breakdown_spd", "laplacian_2d", "csr_of_dense",
    "random_rhs", "SEED_BASE", "reorder", "wavefront_colours", "block_ids", "block_wavefront_colours",
    "block_diagonal_part", "shuffle_within_colours",
]

SEED_BASE = 20220316


@dataclasses.dataclass
class Problem:
    """One SPD matrix in colour-major CSR order plus what a sequence needs.

    rowptr/colind are int32, val float64; columns are sorted inside each row and
    ``colour_ptr[c]:colour_ptr[c+1]`` is the row range of colour ``c``. ``perm[new] = old``
    maps the colour-major index to the natural lexicographic cell index.
    """
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray
    colour_ptr: np.ndarray
    perm: np.ndarray
    dt: float = 0.0
    source: Optional[np.ndarray] = None
    shape: tuple = ()
    h: float = 1.0
    coef: Optional[np.ndarray] = None  # per-cell coefficient, natural order
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def ncolours(self) -> int:
        return len(self.colour_ptr) - 1

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))


def _colour_of(shape):
    idx = np.indices(shape)  # axis order (x, y[, z]); x fastest in the natural numbering
    if len(shape) == 2:
        return ((idx[0] + idx[1]) % 2).astype(np.int64)
    col = np.zeros(shape, dtype=np.int64)
    for ax in range(len(shape)):
        col += (idx[ax] % 2) << ax
    return col


def _natural_index(shape):
    # x fastest: index = x + Nx*(y + Ny*z)
    idx = np.indices(shape)
    lin = np.zeros(shape, dtype=np.int64)
    stride = 1
    for ax in range(len(shape)):
        lin += idx[ax] * stride
        stride *= shape[ax]
    return lin


def fv_diffusion(coef: np.ndarray, h: float, dt: float, name: str = "") -> Problem:
    """Assemble ``A = I/dt + K`` for cell-centred FV diffusion with harmonic-mean faces.

    ``coef`` has shape ``(Nx, Ny[, Nz])`` (axis 0 = x, fastest in the natural numbering).
    ``dt = inf`` gives the steady operator ``K``.
    """
    shape = coef.shape
    d = len(shape)
    n = int(np.prod(shape))
    nat = _natural_index(shape)
    rows, cols, vals = [], [], []
    diag = np.full(shape, 0.0 if not np.isfinite(dt) else 1.0 / dt)
    inv_h2 = 1.0 / (h * h)
    for ax in range(d):
        ka = np.take(coef, np.arange(shape[ax] - 1), axis=ax)
        kb = np.take(coef, np.arange(1, shape[ax]), axis=ax)
        t = 2.0 * ka * kb / (ka + kb) * inv_h2
        ia = np.take(nat, np.arange(shape[ax] - 1), axis=ax).ravel()
        ib = np.take(nat, np.arange(1, shape[ax]), axis=ax).ravel()
        tf = t.ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-tf, -tf]
        # interior faces feed both diagonals
        pad_lo = [(0, 0)] * d
        pad_lo[ax] = (0, 1)
        pad_hi = [(0, 0)] * d
        pad_hi[ax] = (1, 0)
        diag += np.pad(t, pad_lo) + np.pad(t, pad_hi)
        # Dirichlet faces at both ends of this axis
        lo = [slice(None)] * d
        lo[ax] = slice(0, 1)
        hi = [slice(None)] * d
        hi[ax] = slice(shape[ax] - 1, shape[ax])
        diag[tuple(lo)] += 2.0 * coef[tuple(lo)] * inv_h2
        diag[tuple(hi)] += 2.0 * coef[tuple(hi)] * inv_h2
    rows.append(nat.ravel())
    cols.append(nat.ravel())
    vals.append(diag.ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    # colour-major permutation (stable: natural order inside a colour)
    colour = _colour_of(shape).ravel()[np.argsort(nat.ravel())]  # colour by natural index
    perm = np.argsort(colour, kind="stable").astype(np.int64)  # perm[new] = old
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    ncol = int(colour.max()) + 1
    counts = np.bincount(colour, minlength=ncol)
    colour_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    A = sp.csr_matrix((v, (inv[r], inv[c])), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return Problem(n=n, rowptr=A.indptr.astype(np.int32), colind=A.indices.astype(np.int32),
                   val=A.data.astype(np.float64), colour_ptr=colour_ptr, perm=perm, dt=dt,
                   shape=tuple(shape), h=h, coef=coef, name=name)


def reorder(prob: Problem, colour_nat: np.ndarray, name: str = "") -> Problem:
    """The same operator (and source, coefficients) in another multicolour ordering:
    ``colour_nat[k]`` is the colour of natural cell k; rows are colour-major with natural
    order inside a colour. A colour whose rows are coupled is allowed here (a single colour
    is the natural order); the library's own check rejects it."""
    colour_nat = np.asarray(colour_nat, dtype=np.int64).ravel()
    inv = np.empty(prob.n, dtype=np.int64)
    inv[prob.perm] = np.arange(prob.n)
    perm2 = np.argsort(colour_nat, kind="stable").astype(np.int64)  # new -> natural
    q = inv[perm2]                                                   # new -> old row
    A = prob.scipy()[q][:, q].tocsr()
    A.sort_indices()
    ncol = int(colour_nat.max()) + 1
    cp = np.concatenate([[0], np.cumsum(np.bincount(colour_nat, minlength=ncol))]).astype(np.int32)
    out = dataclasses.replace(prob, rowptr=A.indptr.astype(np.int32), colind=A.indices.astype(np.int32),
                              val=A.data.astype(np.float64), colour_ptr=cp, perm=perm2,
                              name=name or prob.name)
    if prob.source is not None:
        out.source = np.ascontiguousarray(prob.source[q])
    return out


def wavefront_colours(shape) -> np.ndarray:
    """Colour x + y (+ z) per natural cell: the wavefronts of natural-order IC(0) on a 5/7-point
    stencil (a row's earlier neighbours all lie on the previous wavefront)."""
    return np.indices(shape).sum(axis=0).ravel(order="F")


def block_ids(shape, b: int) -> np.ndarray:
    """Index of the b^d block holding each natural cell (blocks in natural order)."""
    idx = np.indices(shape)
    nb = [-(-s // b) for s in shape]
    bid = np.zeros(shape, dtype=np.int64)
    stride = 1
    for ax in range(len(shape)):
        bid += (idx[ax] // b) * stride
        stride *= nb[ax]
    return bid.ravel(order="F")


def block_wavefront_colours(shape, b: int) -> np.ndarray:
    """Wavefronts inside b^d blocks (local x + y + z): with the couplings between blocks
    dropped from the preconditioner, IC(0) of each block in natural order (the paper's
    block-Jacobi IC, one block per thread), all blocks advancing together."""
    return (np.indices(shape) % b).sum(axis=0).ravel(order="F")


def block_diagonal_part(prob: Problem, block_nat: np.ndarray) -> Problem:
    """The block-diagonal part of ``prob``'s matrix: entries coupling cells of different blocks
    (``block_nat`` per natural cell) dropped; same ordering."""
    blk = np.asarray(block_nat)[prob.perm]
    A = prob.scipy().tocoo()
    keep = blk[A.row] == blk[A.col]
    B = sp.csr_matrix((A.data[keep], (A.row[keep], A.col[keep])), shape=A.shape)
    B.sort_indices()
    return dataclasses.replace(prob, rowptr=B.indptr.astype(np.int32), colind=B.indices.astype(np.int32),
                               val=B.data.astype(np.float64), name=prob.name + "_blockdiag")


def square_inclusions(N: int, count: int, size: int, value: float, rng) -> np.ndarray:
    """Background 1 with ``count`` non-overlapping ``size x size`` squares of ``value``."""
    coef = np.ones((N, N))
    placed = []
    while len(placed) < count:
        x0, y0 = rng.integers(0, N - size + 1, size=2)
        if any(abs(x0 - a) < size and abs(y0 - b) < size for a, b in placed):
            continue
        placed.append((x0, y0))
        coef[x0:x0 + size, y0:y0 + size] = value
    return coef


def sphere_inclusions(N: int, count: int, rmin: float, rmax: float, value: float, rng) -> np.ndarray:
    """Background 1 with ``count`` non-overlapping balls (radius in cells, fully inside)."""
    coef = np.ones((N, N, N))
    centres = []
    ctr = np.indices((N, N, N)).astype(np.float64) + 0.5
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place inclusions")
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(r, N - r, size=3)
        if any(np.linalg.norm(c - c2) < r + r2 for c2, r2 in centres):
            continue
        centres.append((c, r))
        lo = np.maximum(np.floor(c - r).astype(int), 0)
        hi = np.minimum(np.ceil(c + r).astype(int) + 1, N)
        sub = tuple(slice(lo[a], hi[a]) for a in range(3))
        d2 = sum((ctr[a][sub] - c[a]) ** 2 for a in range(3))
        coef[sub][d2 <= r * r] = value
    return coef


def gaussian_source(shape, sigma: float = 0.1, centre: float = 0.5) -> np.ndarray:
    """Fixed spatial Gaussian bump on cell centres, natural order."""
    N = shape[0]
    x = (np.indices(shape) + 0.5) / N
    d2 = sum((x[a] - centre) ** 2 for a in range(len(shape)))
    return np.exp(-d2 / (2.0 * sigma * sigma))


def smooth_gaussian_field(shape, corr_cells: float, rng) -> np.ndarray:
    """White noise convolved with a Gaussian of std ``corr_cells`` cells, unit variance."""
    from scipy.ndimage import gaussian_filter
    w = rng.standard_normal(shape)
    f = gaussian_filter(w, sigma=corr_cells, mode="wrap")
    f -= f.mean()
    return f / f.std()


def _finish(p: Problem, src_nat: np.ndarray) -> Problem:
    p.source = np.ascontiguousarray(src_nat.ravel(order="F")[p.perm])
    return p


def config_c1(seed: int = SEED_BASE + 0) -> Problem:
    """2D 64x64 5-point FV, 4 seeded 6x6 inclusions of 1e3, red-black, dt = 1e-2,
    source uniform in [0,1) drawn once per sequence."""
    rng = np.random.default_rng(seed)
    N = 64
    coef = square_inclusions(N, 4, 6, 1e3, rng)
    p = fv_diffusion(coef, 1.0 / N, 1e-2, name="fv5_64x64_redblack")
    return _finish(p, rng.uniform(0.0, 1.0, size=(N, N)))


def config_c2(N: int = 128, seed: int = SEED_BASE + 1, count: int = 16, rmin: float = 4.0,
              rmax: float = 8.0, value: float = 1e5, dt: float = 1e-3) -> Problem:
    """3D 7-point FV on N^3, ``count`` balls of radius rmin..rmax cells with coefficient
    ``value``, 8-colour ordering, dt = 1e-3, Gaussian source (centre 0.5, sigma 0.1)."""
    rng = np.random.default_rng(seed)
    coef = sphere_inclusions(N, count, rmin, rmax, value, rng)
    p = fv_diffusion(coef, 1.0 / N, dt, name=f"fv7_{N}cube_8colour")
    return _finish(p, gaussian_source((N, N, N)))


def config_c4(N: int = 128, seed: int = SEED_BASE + 3, corr: float = 4.0):
    """3D 7-point steady FV with k = exp(theta), theta ~ N(0,1) smoothed over ``corr``
    cells (renormalised to unit variance). Returns (problem, theta, x_target)."""
    rng = np.random.default_rng(seed)
    theta = smooth_gaussian_field((N, N, N), corr, rng)
    p = fv_diffusion(np.exp(theta), 1.0 / N, np.inf, name=f"fv7_{N}cube_lognormal")
    p = _finish(p, gaussian_source((N, N, N)))
    x_target = rng.standard_normal(p.n) * 1e-3
    return p, theta, x_target


def _colour_major_csr(cols_nat: np.ndarray, vals: np.ndarray, shape, dt: float, h: float, name: str,
                      coef=None) -> Problem:
    """CSR in the 8-colour (2-colour in 2D) order from a dense per-node stencil table:
    ``cols_nat[c, s]`` is the natural index of the s-th neighbour of natural node c (-1 when
    absent) and ``vals[c, s]`` its value. Columns are sorted inside each row."""
    n = int(np.prod(shape))
    colour = _colour_of(shape).ravel(order="F")  # natural order, x fastest
    perm = np.argsort(colour, kind="stable").astype(np.int64)  # perm[row] = natural node
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    counts = np.bincount(colour, minlength=int(colour.max()) + 1)
    colour_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    big = np.iinfo(np.int32).max
    cr = cols_nat[perm]
    vr = vals[perm]
    valid = cr >= 0
    cols = np.where(valid, inv[np.where(valid, cr, 0)], big).astype(np.int32)
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    vr = np.take_along_axis(vr, order, axis=1)
    keep = cols != big
    rowptr = np.concatenate([[0], np.cumsum(keep.sum(axis=1))]).astype(np.int32)
    return Problem(n=n, rowptr=rowptr, colind=np.ascontiguousarray(cols[keep]),
                   val=np.ascontiguousarray(vr[keep]), colour_ptr=colour_ptr, perm=perm, dt=dt,
                   shape=tuple(shape), h=h, coef=coef, name=name)


def fe27_diffusion(kelem: np.ndarray, aniso=(1.0, 1.0, 1e-3), dt: float = 1e-3, name: str = "") -> Problem:
    """Q1 (trilinear) finite elements on the unit cube, homogeneous Dirichlet boundary.

    ``kelem`` holds one coefficient per element, shape (E, E, E) with axis 0 = x; the
    unknowns are the N = E - 1 interior nodes per axis, h = 1/E. The element tensor is
    ``k_e diag(aniso)``; on a cube of side h the stiffness of axis d is
    ``k_e aniso_d (h/36) (K1 (x) M1 (x) M1)`` with K1 = [[1,-1],[-1,1]] along d and
    M1 = [[2,1],[1,2]] along the other two axes. A = I/dt + K / h^3 (27-point stencil).
    """
    E = kelem.shape[0]
    N = E - 1
    h = 1.0 / E
    shape = (N, N, N)
    n = N ** 3
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]])
    idx = np.indices(shape)  # node (i, j, k) -> interior node index 0..N-1 along each axis
    nat = (idx[0] + N * (idx[1] + N * idx[2]))
    offsets = [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)]
    cols = np.full((n, 27), -1, dtype=np.int64)
    vals = np.zeros((n, 27))
    inv_dt = 0.0 if not np.isfinite(dt) else 1.0 / dt
    scale = (h / 36.0) / h ** 3
    for s, o in enumerate(offsets):
        v = np.zeros(shape)
        # elements holding both the node p and its neighbour p + o: along an axis with o_d = 0
        # the two elements left and right of p, otherwise the one between them; element e
        # spans the nodes e, e + 1 of the full grid (interior node i is full-grid node i + 1)
        choices = [(-1, 0) if od == 0 else ((0,) if od == 1 else (-1,)) for od in o]
        for e0 in choices[0]:
            for e1 in choices[1]:
                for e2 in choices[2]:
                    e_off = (e0, e1, e2)
                    a = [-eo for eo in e_off]          # local index of p in the element
                    b = [a[d] + o[d] for d in range(3)]  # local index of p + o
                    cf = (aniso[0] * k1[a[0], b[0]] * m1[a[1], b[1]] * m1[a[2], b[2]]
                          + aniso[1] * m1[a[0], b[0]] * k1[a[1], b[1]] * m1[a[2], b[2]]
                          + aniso[2] * m1[a[0], b[0]] * m1[a[1], b[1]] * k1[a[2], b[2]])
                    # element index of interior node i (full-grid node i + 1) is i + 1 + e_off
                    sl = tuple(slice(1 + e_off[d], 1 + e_off[d] + N) for d in range(3))
                    v += cf * kelem[sl]
        v *= scale
        if o == (0, 0, 0):
            v += inv_dt
        ok = np.ones(shape, dtype=bool)
        for d in range(3):
            q = idx[d] + o[d]
            ok &= (q >= 0) & (q < N)
        qn = nat + o[0] + N * (o[1] + N * o[2])
        cols[:, s] = np.where(ok, qn, -1).ravel(order="F")
        vals[:, s] = np.where(ok, v, 0.0).ravel(order="F")
    return _colour_major_csr(cols, vals, shape, dt, h, name or f"fe27_{N}cube")


def config_c3(N: int = 192, seed: int = SEED_BASE + 2, sigma: float = 2.0, corr: float = 8.0,
              dt: float = 1e-3) -> Problem:
    """3D 27-point Q1 FE on N^3 interior nodes, tensor diag(1, 1, 1e-3) times a log-normal
    per-element coefficient (sigma 2, correlation length 8 elements), dt = 1e-3 (backward
    Euler, as C2), Gaussian source (centre 0.5, sigma 0.1) at the nodes."""
    rng = np.random.default_rng(seed)
    E = N + 1
    kelem = np.exp(sigma * smooth_gaussian_field((E, E, E), corr, rng))
    p = fe27_diffusion(kelem, dt=dt, name=f"fe27_{N}cube_aniso_lognormal")
    x = (np.indices((N, N, N)) + 1.0) / E
    src = np.exp(-sum((x[a] - 0.5) ** 2 for a in range(3)) / (2.0 * 0.1 * 0.1))
    return _finish(p, src)


def config_c5(N: int = 256, seed: int = SEED_BASE + 4, count: int = 64, rmin: float = 8.0,
              rmax: float = 16.0, value: float = 1e6, dt: float = 1e-3) -> Problem:
    """C2's recipe at 256^3 with 64 balls of coefficient 1e6 (radius 8-16 cells: C2's 4-8
    at twice the resolution)."""
    return config_c2(N=N, seed=seed, count=count, rmin=rmin, rmax=rmax, value=value, dt=dt)


def small_3d(N: int, seed: int, count: int = 2, rmin: float = 1.5, rmax: float = 2.5,
             value: float = 1e3, dt: float = 1e-3) -> Problem:
    """A reduced C2-like problem for parity tests (odd N gives ragged colour sizes)."""
    rng = np.random.default_rng(seed)
    if N < 7:  # too small for non-overlapping balls: one small inclusion at most
        count, rmin, rmax = min(count, 1), min(rmin, N / 4), min(rmax, N / 4)
    coef = sphere_inclusions(N, count, rmin, rmax, value, rng) if count else np.ones((N, N, N))
    p = fv_diffusion(coef, 1.0 / N, dt, name=f"fv7_{N}cube")
    return _finish(p, gaussian_source((N, N, N)))


def shuffle_within_colours(p: Problem, seed: int) -> Problem:
    """The same operator with the rows of every colour in a seeded random order (still a
    valid colouring: rows of one colour are uncoupled). Scatters the neighbours of a 32-row
    slice, so the FP32 copy keeps (value, column) pairs instead of per-slice column bases."""
    rng = np.random.default_rng(seed)
    cp = np.asarray(p.colour_ptr)
    q = np.concatenate([cp[c] + rng.permutation(cp[c + 1] - cp[c]) for c in range(len(cp) - 1)])  # new -> old
    A = p.scipy()[q][:, q].tocsr()
    A.sort_indices()
    out = dataclasses.replace(p, rowptr=A.indptr.astype(np.int32), colind=A.indices.astype(np.int32),
                              val=A.data.astype(np.float64), perm=np.asarray(p.perm)[q], name=p.name + "_shuffled")
    out.source = np.ascontiguousarray(p.source[q])
    return out


def random_rhs(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=n)


# ---- tiny dense-defined test matrices (for the pins) ----

def random_spd_dense(eigs: np.ndarray, seed: int) -> np.ndarray:
    """``Q diag(eigs) Q^T`` with a seeded random orthogonal Q."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((len(eigs), len(eigs))))
    a = (q * eigs) @ q.T
    return 0.5 * (a + a.T)


def csr_of_dense(a: np.ndarray, ncolours: int = 1) -> Problem:
    """Dense SPD matrix as a CSR problem with a single colour (or the given count of
    equal contiguous colour blocks, valid only when the blocks have no internal edges)."""
    n = a.shape[0]
    m = sp.csr_matrix(a)
    m.sort_indices()
    cp = np.linspace(0, n, ncolours + 1).astype(np.int32)
    return Problem(n=n, rowptr=m.indptr.astype(np.int32), colind=m.indices.astype(np.int32),
                   val=m.data.astype(np.float64), colour_ptr=cp, perm=np.arange(n))


def ic0_breakdown_spd(n: int = 24, seed: int = 7, margin: float = 1e-3) -> Problem:
    """A sparse SPD matrix that is not an M-matrix (off-diagonal entries of both signs, about
    15 % density), shifted so that its smallest eigenvalue is ``margin``; one row per colour.
    With the defaults IC(0) of A meets a non-positive pivot and succeeds on A + s diag(A)
    only from s = 8e-3."""
    rng = np.random.default_rng(seed)
    b = sp.random(n, n, density=0.15, random_state=rng, data_rvs=lambda k: rng.uniform(-1, 1, k)).toarray()
    s = b + b.T
    np.fill_diagonal(s, 0.0)
    a = s + np.eye(n) * (margin - np.linalg.eigvalsh(s).min())
    return csr_of_dense(a, ncolours=n)


def laplacian_1d(n: int) -> Problem:
    """tridiag(-1, 2, -1) of order n, red-black ordered (odd points first)."""
    a = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    colour = np.arange(n) % 2
    perm = np.argsort(colour, kind="stable")
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    ap = a[perm][:, perm].tocsr()
    ap.sort_indices()
    counts = np.bincount(colour, minlength=2)
    cp = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return Problem(n=n, rowptr=ap.indptr.astype(np.int32), colind=ap.indices.astype(np.int32),
                   val=ap.data.astype(np.float64), colour_ptr=cp, perm=perm, name="lap1d")


def laplacian_2d(N: int) -> Problem:
    """5-point Laplacian 4,-1 on an N x N grid (unit spacing), red-black ordered."""
    coef = np.ones((N, N))
    p = fv_diffusion(coef, 1.0, np.inf, name="lap2d")
    # fv_diffusion with h=1, k=1 gives interior faces 1 and boundary faces 2: rescale to the
    # textbook stencil by rebuilding the diagonal as 4 on every row.
    A = p.scipy().tolil()
    for i in range(p.n):
        A[i, i] = 4.0
    A = A.tocsr()
    A.sort_indices()
    p.rowptr = A.indptr.astype(np.int32)
    p.colind = A.indices.astype(np.int32)
    p.val = A.data.astype(np.float64)
    return p

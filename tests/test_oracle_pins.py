"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties an oracle routine to something other than itself: the paper's worked
example, a closed form, a theorem (exact CG termination, Cauchy interlacing, the spectral
statements of Section 4.1), a dense direct solve, or brute force on a tiny input.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- sampling method A

def _golden_sampling(name="sampling_method_a.txt"):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            v = [int(t) for t in line.split()]
            rows.append((v[0], v[1], v[2:]))
    return rows


@pytest.mark.parametrize("m,N,kept", _golden_sampling())
def test_sampling_a_worked_example(m, N, kept):
    """Section 4.3: m = 4 and convergence at 1000 keep iterations 256, 384, 512, 768."""
    for lmax in (None, 8, 12):  # any l_max with m^l_max > N_max gives the same schedule
        got = sorted(oracle.sampling_a_schedule(m, N, lmax).tolist())
        assert got == kept


@pytest.mark.parametrize("m,N,kept", _golden_sampling("sampling_method_a_sign.txt"))
def test_sampling_a_alternating_sign(m, N, kept):
    """Appendix A, Algorithm alg1: i_t carries the alternating sign (-1)^l. The rows were
    worked by hand from the algorithm for (m, N) where the signed and the unsigned sums
    keep different iterations (the derivations are in the file's header)."""
    for lmax in (None, 6, 9):
        got = sorted(oracle.sampling_a_schedule(m, N, lmax).tolist())
        assert got == kept


def test_sampling_a_in_solve_follows_the_alternating_sign():
    """The same rule inside the oracle's solve: a 3-slot sampled ICCG run keeps the
    iterations the hand-checked schedule gives for its iteration count, which with m = 3
    differ from the unsigned reading's."""
    p = wl.config_c1()
    out = oracle.System(p, oracle.IC0(p)).solve(p.source, tol=1e-8, sample_m=3)
    N = out["iters"]
    want = oracle.sampling_a_schedule(3, N, oracle.default_lmax(3, 20000))
    assert sorted(out["sample_iter"].tolist()) == sorted(want.tolist())
    unsigned = _unsigned_schedule(3, N)
    assert sorted(unsigned) != sorted(want.tolist()), "choose a run where the readings differ"


def _unsigned_schedule(m, N):
    """Algorithm alg1 with every term of i_t added (the reading the sign rows exclude)."""
    h, slots = 1, [0] * m
    for i in range(1, N):
        if i % h:
            continue
        it, q = 0, i - 1
        while q:
            it += q
            q //= m
        slots[it % m] = i
        if i == h * m:
            h *= 2
    return slots


def test_sampling_a_brute_force_properties():
    """Every slot is filled once N > m, the kept iterations are distinct, and none is the
    converging iteration (the convergence check precedes the sampling step)."""
    for m in (2, 3, 5, 8, 16):
        for N in (m + 1, 50, 333, 1000, 4097):
            s = oracle.sampling_a_schedule(m, N)
            assert (s > 0).all() and len(set(s.tolist())) == m and s.max() < N


@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_sampling_a_interval_property(m):
    """Section 4.3 (the paragraph commented out beside the worked example): the kept
    iterations are spaced 2^d or 2^(d+1) apart, d < log2(N/m) <= d+1."""
    for N in range(2 * m + 1, 3000, 13):
        kept = np.sort(oracle.sampling_a_schedule(m, N))
        d = int(np.ceil(np.log2(N / m))) - 1
        gaps = np.diff(kept)
        assert np.all((gaps == 2 ** d) | (gaps == 2 ** (d + 1))), (N, kept)


def test_sampling_inside_solver_matches_schedule():
    p = wl.config_c1()
    out = oracle.System(p, oracle.IC0(p)).solve(p.source, tol=1e-8, sample_m=8)
    want = oracle.sampling_a_schedule(8, out["iters"], oracle.default_lmax(8, 20000))
    assert sorted(out["sample_iter"].tolist()) == sorted(want.tolist())


# ---------------------------------------------------------------- IC(0)

def test_ic0_is_exact_cholesky_on_full_pattern():
    """With a full pattern there is no dropped fill: IC(0) is the Cholesky factor."""
    a = wl.random_spd_dense(np.linspace(1.0, 30.0, 12), seed=3)
    p = wl.csr_of_dense(a)
    ic = oracle.IC0(p)
    assert ic.shift == 0.0
    np.testing.assert_allclose(ic.dense_L(), np.linalg.cholesky(a), rtol=1e-12, atol=1e-12)


def _random_sparse_spd(n, density, seed):
    rng = np.random.default_rng(seed)
    b = sp.random(n, n, density=density, random_state=rng, data_rvs=lambda k: -rng.uniform(0.1, 1, k))
    s = (b + b.T).tocsr()
    s.setdiag(0)
    s.eliminate_zeros()
    d = np.asarray(abs(s).sum(axis=1)).ravel() + 1.0
    a = (s + sp.diags(d)).tocsr()
    a.sort_indices()
    return a


@pytest.mark.parametrize("kind", ["fv7", "random_with_triangles"])
def test_ic0_reproduces_A_on_its_pattern(kind):
    """Defining property of IC(0): (L L^T)_ij = a_ij for every (i, j) in tril(A)."""
    if kind == "fv7":
        p = wl.small_3d(5, seed=1)
    else:
        a = _random_sparse_spd(60, 0.08, seed=4)
        p = wl.Problem(n=60, rowptr=a.indptr.astype(np.int32), colind=a.indices.astype(np.int32),
                       val=a.data, colour_ptr=np.array([0, 60], np.int32), perm=np.arange(60))
    ic = oracle.IC0(p)
    L = sp.csr_matrix((ic.Lva, ic.Lci, ic.Lrp), shape=(p.n, p.n))
    LLt = (L @ L.T).tocsr()
    A = sp.tril(p.scipy()).tocoo()
    np.testing.assert_allclose(np.asarray(LLt[A.row, A.col]).ravel(), A.data, rtol=1e-12, atol=1e-9)
    if kind == "random_with_triangles":
        # the pattern has triangles, so L L^T differs from A somewhere off the pattern
        assert abs(LLt - p.scipy()).max() > 1e-8


def test_ic0_shift_rule_on_indefinite_pivot():
    """A matrix whose IC(0) breaks down is factorised after the diagonal shift."""
    a = np.array([[1.0, 0.9, 0.9], [0.9, 1.0, -0.9], [0.9, -0.9, 1.0]])  # indefinite
    p = wl.csr_of_dense(a + 0.0)
    with pytest.raises(ArithmeticError):
        oracle.IC0(p, max_tries=1)
    ic = oracle.IC0(p, max_tries=40)
    assert ic.shift > 0


@pytest.mark.parametrize("which", ["c1", "small3d"])
def test_ic_apply_is_M_inverse(which):
    """Colour-ordered substitutions give z = (L L^T)^{-1} r (dense direct solve)."""
    p = wl.config_c1() if which == "c1" else wl.small_3d(7, seed=2)
    ic = oracle.IC0(p)
    r = np.random.default_rng(5).standard_normal(p.n)
    z = ic.apply(r)
    L = sp.csr_matrix((ic.Lva, ic.Lci, ic.Lrp), shape=(p.n, p.n)).tocsc()
    y = spla.spsolve_triangular(L.tocsr(), r, lower=True)
    z_ref = spla.spsolve_triangular(L.T.tocsr(), y, lower=False)
    np.testing.assert_allclose(z, z_ref, rtol=1e-11, atol=1e-13 * np.abs(z_ref).max())


def test_colouring_has_no_intra_colour_edges():
    for p in (wl.config_c1(), wl.small_3d(6, seed=0), wl.laplacian_1d(9), wl.laplacian_2d(5)):
        A = p.scipy().tocoo()
        col = np.searchsorted(p.colour_ptr, np.arange(p.n), side="right") - 1
        off = A.row != A.col
        assert not np.any(col[A.row[off]] == col[A.col[off]])


# ---------------------------------------------------------------- CG

@pytest.mark.parametrize("k", [2, 4, 7])
def test_cg_terminates_in_k_steps(k):
    """CG on a matrix with k distinct eigenvalues ends in at most k iterations."""
    a = wl.random_spd_dense(np.repeat(np.linspace(1.0, 100.0, k), 5), seed=k)
    p = wl.csr_of_dense(a)
    b = np.random.default_rng(k).standard_normal(p.n)
    out = oracle.System(p, None).solve(b, tol=1e-12, maxit=100)
    assert out["iters"] <= k and out["relres"] <= 1e-12
    np.testing.assert_allclose(out["x"], np.linalg.solve(a, b), rtol=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_cg_reaches_1e12_within_n(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 21))
    a = wl.random_spd_dense(np.linspace(1.0, 1e3, n), seed=seed)
    p = wl.csr_of_dense(a)
    b = rng.standard_normal(n)
    out = oracle.System(p, None).solve(b, tol=1e-12, maxit=10 * n)
    assert out["iters"] <= n


def test_iccg_solves_the_system():
    p = wl.small_3d(9, seed=3)
    out = oracle.System(p, oracle.IC0(p)).solve(p.source, tol=1e-10)
    A = p.scipy()
    x_ref = spla.spsolve(A.tocsc(), p.source)
    assert np.linalg.norm(p.source - A @ out["x"]) <= 1.01e-10 * np.linalg.norm(p.source)
    np.testing.assert_allclose(out["x"], x_ref, rtol=1e-7, atol=1e-9 * np.abs(x_ref).max())
    assert out["relres"] == pytest.approx(np.linalg.norm(p.source - A @ out["x"]) / np.linalg.norm(p.source), rel=1e-4)


def test_zero_rhs_and_converged_start():
    p = wl.small_3d(4, seed=0)
    s = oracle.System(p, oracle.IC0(p))
    out = s.solve(np.zeros(p.n), x0=np.ones(p.n))
    assert out["iters"] == 0 and np.all(out["x"] == 0)
    x_ref = spla.spsolve(p.scipy().tocsc(), p.source)
    out = s.solve(p.source, x0=x_ref, tol=1e-8)
    assert out["iters"] == 0


# ---------------------------------------------------------------- deflation / SC with exact eigenvectors

def _isolated_small(n=64, m=4, k=6, seed=7):
    small = np.array([1e-4, 3e-4, 7e-4, 1.5e-3])[:m]
    big = np.repeat(np.linspace(1.0, 50.0, k), (n - m) // k)
    ev = np.concatenate([small, big])
    a = wl.random_spd_dense(ev, seed=seed)
    return a, ev, wl.csr_of_dense(a)


def test_deflation_with_exact_eigenvectors():
    """Section 4.1: deflating the m small eigenvectors leaves the k distinct others, so
    deflated CG (M = I) ends in <= k iterations while plain CG needs more; W^T r_i = 0."""
    a, ev, p = _isolated_small()
    w, V = np.linalg.eigh(a)
    aux = oracle.Aux.from_basis(p, V[:, :4])
    b = np.random.default_rng(1).standard_normal(p.n)
    plain = oracle.System(p, None).solve(b, tol=1e-10, maxit=500)
    defl = oracle.System(p, None, oracle.DEFLATION, aux).solve(b, tol=1e-10, maxit=500)
    assert defl["iters"] <= 6 < plain["iters"]
    assert defl["wtr"].max() <= 1e-12
    assert np.linalg.norm(b - a @ defl["x"]) <= 1.01e-10 * np.linalg.norm(b)


def test_subspace_correction_shifts_small_eigenvalue_by_one():
    """Section 4.1: with M = I and W = [u_s], M_sc^{-1} A has lambda_s + 1 and otherwise
    the spectrum of A."""
    a, ev, p = _isolated_small(m=1)
    w, V = np.linalg.eigh(a)
    aux = oracle.Aux.from_basis(p, V[:, :1])
    s = oracle.System(p, None, oracle.SUBSPACE_CORRECTION, aux)
    op = np.column_stack([s.precond(a[:, j]) for j in range(p.n)])
    got = np.sort(np.linalg.eigvals(op).real)
    want = np.sort(np.concatenate([[w[0] + 1.0], w[1:]]))
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------- Lanczos condition estimate

def test_lanczos_1d_laplacian_closed_form():
    """Plain CG on tridiag(-1,2,-1), n = 50: the Lanczos extremes are 2 - 2cos(k pi/51)."""
    n = 50
    p = wl.laplacian_1d(n)
    b = np.random.default_rng(0).standard_normal(n)
    out = oracle.System(p, None).solve(b, tol=1e-14, maxit=200)
    lmin, lmax, kappa = oracle.estimate_cond(out["alpha"], out["beta"])
    assert lmin == pytest.approx(2 - 2 * np.cos(np.pi / (n + 1)), rel=1e-8)
    assert lmax == pytest.approx(2 - 2 * np.cos(n * np.pi / (n + 1)), rel=1e-8)


def test_lanczos_2d_laplacian_closed_form():
    N = 10
    p = wl.laplacian_2d(N)
    b = np.random.default_rng(1).standard_normal(p.n)
    out = oracle.System(p, None).solve(b, tol=1e-14, maxit=500)
    lmin, lmax, _ = oracle.estimate_cond(out["alpha"], out["beta"])
    c = np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    lam = 4 - 2 * c[:, None] - 2 * c[None, :]
    assert lmin == pytest.approx(lam.min(), rel=1e-8)
    assert lmax == pytest.approx(lam.max(), rel=1e-8)


def test_lanczos_preconditioned_bounds():
    """With IC(0) the estimate brackets nothing outside the spectrum of M^{-1} A."""
    p = wl.small_3d(5, seed=1)
    ic = oracle.IC0(p)
    b = np.random.default_rng(0).standard_normal(p.n)
    out = oracle.System(p, ic).solve(b, tol=1e-14, maxit=1000)
    lmin, lmax, _ = oracle.estimate_cond(out["alpha"], out["beta"])
    L = ic.dense_L()
    Li = np.linalg.inv(L)
    ev = np.linalg.eigvalsh(Li @ p.scipy().toarray() @ Li.T)
    assert ev.min() * (1 - 1e-8) <= lmin and lmax <= ev.max() * (1 + 1e-8)
    assert lmax == pytest.approx(ev.max(), rel=1e-6)
    assert lmin == pytest.approx(ev.min(), rel=1e-6)


# ---------------------------------------------------------------- auxiliary matrix

# ---------------------------------------------------------------- diagonal scaling

def test_diag_scaled_laplacian_closed_form():
    """tridiag(-1, 2, -1) scaled by its diagonal is tridiag(-1/2, 1, -1/2): unit diagonal and
    eigenvalues 1 - cos(k pi/(n+1)); CG on it reaches those extremes in its Lanczos matrix."""
    n = 40
    p = wl.laplacian_1d(n)
    ps, d = oracle.diag_scale(p)
    np.testing.assert_array_equal(d, np.full(n, 1 / np.sqrt(2.0)))
    A = ps.scipy().toarray()
    np.testing.assert_allclose(np.diag(A), 1.0, rtol=1e-15)
    np.testing.assert_array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(ev, np.sort(1 - np.cos(np.arange(1, n + 1) * np.pi / (n + 1))), atol=1e-14)
    out = oracle.System(ps, None).solve(np.random.default_rng(2).standard_normal(n), tol=1e-14, maxit=200)
    lmin, lmax, _ = oracle.estimate_cond(out["alpha"], out["beta"])
    assert lmin == pytest.approx(1 - np.cos(np.pi / (n + 1)), rel=1e-8)
    assert lmax == pytest.approx(1 - np.cos(n * np.pi / (n + 1)), rel=1e-8)


def test_diag_scaled_matrix_symmetric_unit_diagonal():
    """On variable coefficients (contrast 1e3): A^ keeps A's symmetry, has a unit diagonal,
    and equals D^-1/2 A D^-1/2 formed as a dense product."""
    p = wl.small_3d(7, seed=5)
    ps, d = oracle.diag_scale(p)
    A = p.scipy().toarray()
    As = ps.scipy().toarray()
    np.testing.assert_allclose(As, As.T, rtol=1e-15, atol=0)
    np.testing.assert_allclose(np.diag(As), 1.0, rtol=4.5e-16)  # (a d) d: two roundings
    Dm = np.diag(1.0 / np.sqrt(np.diag(A)))
    np.testing.assert_allclose(As, Dm @ A @ Dm, rtol=1e-15, atol=1e-16)


def test_ic0_is_invariant_under_diag_scaling():
    """IC(0) commutes with symmetric diagonal scaling: the factor of D^-1/2 A D^-1/2 is
    D^-1/2 L (every product on the pattern scales by d_i d_j), so ICCG takes the same
    iterations on A x = b and on A^ x^ = d b, and d x^ solves A x = b."""
    p = wl.small_3d(7, seed=5)
    ps, d = oracle.diag_scale(p)
    L = oracle.IC0(p).dense_L()
    Ls = oracle.IC0(ps).dense_L()
    np.testing.assert_allclose(Ls, d[:, None] * L, rtol=1e-12, atol=1e-14 * np.abs(Ls).max())
    b = p.source
    out = oracle.System(p, oracle.IC0(p)).solve(b, tol=1e-10)
    outs = oracle.System(ps, oracle.IC0(ps)).solve(d * b, tol=1e-10)
    assert abs(out["iters"] - outs["iters"]) <= 1
    x = d * outs["x"]
    assert np.linalg.norm(b - p.scipy() @ x) <= 1e-8 * np.linalg.norm(b)


def test_diag_scaling_rejects_nonpositive_diagonal():
    p = wl.laplacian_1d(6)
    bad = wl.laplacian_1d(6)
    bad.val = p.val.copy()
    rows = np.repeat(np.arange(6), np.diff(p.rowptr))
    bad.val[np.flatnonzero(rows == p.colind)[2]] = -1.0
    with pytest.raises(ValueError):
        oracle.diag_scale(bad)


# ---------------------------------------------------------------- other IC orderings

def test_wavefront_ic0_is_natural_order_ic0():
    """Rows on one wavefront x+y+z are uncoupled and every earlier neighbour of a row lies on
    an earlier wavefront, so IC(0) in wavefront order is natural-order IC(0) up to the
    symmetric permutation: M^-1 r agrees mapped to natural order, and ICCG takes the same
    iterations to the same solution. (The natural order gives every cell its own colour, so
    the oracle's sweeps take the rows one by one.)"""
    p = wl.small_3d(7, seed=5)
    pn = wl.reorder(p, np.arange(p.n))
    pw = wl.reorder(p, wl.wavefront_colours(p.shape))
    assert pw.ncolours == 3 * 7 - 2
    r = np.random.default_rng(8).standard_normal(p.n)  # natural order
    zn = oracle.IC0(pn).apply(r[pn.perm])
    zw = oracle.IC0(pw).apply(r[pw.perm])
    z_nat_n, z_nat_w = np.empty(p.n), np.empty(p.n)
    z_nat_n[pn.perm], z_nat_w[pw.perm] = zn, zw
    np.testing.assert_allclose(z_nat_w, z_nat_n, rtol=1e-12, atol=1e-14 * np.abs(z_nat_n).max())
    on = oracle.System(pn, oracle.IC0(pn)).solve(pn.source, tol=1e-10)
    ow = oracle.System(pw, oracle.IC0(pw)).solve(pw.source, tol=1e-10)
    assert on["iters"] == ow["iters"]
    xn, xw = np.empty(p.n), np.empty(p.n)
    xn[pn.perm], xw[pw.perm] = on["x"], ow["x"]
    np.testing.assert_allclose(xw, xn, rtol=1e-12, atol=1e-12 * np.abs(xn).max())
    # and multicolour IC(0) is a different (weaker) preconditioner on this problem
    om = oracle.System(p, oracle.IC0(p)).solve(p.source, tol=1e-10)
    assert om["iters"] > on["iters"]


def test_block_jacobi_ic0_factors_each_block_alone():
    """Block-Jacobi IC (one IC(0) per block, couplings between blocks dropped): M^-1 r on each
    block equals the IC(0) solve of that block's submatrix by itself, and the blocks share
    no entry of the factor."""
    p = wl.small_3d(8, seed=6)
    b = 4
    bid = wl.block_ids(p.shape, b)
    pb = wl.reorder(p, wl.block_wavefront_colours(p.shape, b))
    P = wl.block_diagonal_part(pb, bid)
    assert P.nnz < pb.nnz
    ic = oracle.IC0(P)
    L = ic.dense_L()
    brow = bid[pb.perm]
    assert np.all(L[brow[:, None] != brow[None, :]] == 0)
    r = np.random.default_rng(9).standard_normal(p.n)
    z = ic.apply(r)
    Pd = P.scipy().toarray()
    for blk in np.unique(brow):
        rows = np.flatnonzero(brow == blk)
        sub = wl.csr_of_dense(Pd[np.ix_(rows, rows)], ncolours=len(rows))  # one row per colour
        zs = oracle.IC0(sub).apply(r[rows])
        np.testing.assert_allclose(z[rows], zs, rtol=1e-12, atol=1e-14 * np.abs(zs).max())


# ---------------------------------------------------------------- power method (Section 5.4)

@pytest.mark.parametrize("k", [0, 1, 2, 5, 30])
def test_power_method_diagonal_closed_form(k):
    """On D = diag(d) the k-th power vector is D^k v0 / ||D^k v0|| and lambda_max is
    sum d^(2k+1) v0^2 / sum d^(2k) v0^2 (written out here, not by the oracle's steps)."""
    d = np.linspace(0.5, 3.0, 40)
    p = wl.csr_of_dense(np.diag(d))
    v0 = np.random.default_rng(11).standard_normal(40)
    lam, v = oracle.power_method(p, v0, k)
    w = v0 * d ** k
    assert lam == pytest.approx(np.sum(d ** (2 * k + 1) * v0 ** 2) / np.sum(d ** (2 * k) * v0 ** 2), rel=1e-13)
    np.testing.assert_allclose(v, w / np.linalg.norm(w), rtol=1e-12, atol=1e-15)


def test_power_method_2d_laplacian_top_eigenvalue_and_monotone():
    """5-point Laplacian on 8 x 8: the estimate reaches 4 + 4 cos(pi/9) (the simple top
    eigenvalue; the next ratio is 0.955, so 400 steps leave ~1e-16), and the Rayleigh
    quotients of the power vectors of an SPD matrix never decrease (the moment sequence
    (v0, A^j v0) is log-convex) and never pass the top eigenvalue."""
    p = wl.laplacian_2d(8)
    v0 = np.random.default_rng(12).standard_normal(p.n)
    top = 4 + 4 * np.cos(np.pi / 9)
    lam, v = oracle.power_method(p, v0, 400)
    assert lam == pytest.approx(top, rel=1e-12)
    c = np.cos(np.arange(1, 9) * np.pi / 9)
    lam_sorted = np.sort((4 - 2 * c[:, None] - 2 * c[None, :]).ravel())
    assert lam_sorted[-2] < top * 0.96
    seq = [oracle.power_method(p, v0, k)[0] for k in range(40)]
    assert all(b >= a * (1 - 1e-15) for a, b in zip(seq, seq[1:]))
    assert max(seq) <= top * (1 + 1e-15)


@pytest.mark.parametrize("precond", [False, True])
def test_pcg_cond_estimate_brackets_and_approximates_kappa(precond):
    """Algorithm PCG-con: lambda_max from the power method lies at or below the top
    eigenvalue, the smallest Ritz value of the sampled errors at or above the bottom one, so
    the estimate never exceeds kappa(A). The power method takes one step per CG iteration.
    Without a preconditioner the sampled errors are rich in the bottom eigenvectors of A
    itself: after 101 steps lambda_max is exact to 1e-6 and lambda_min within 10 % on this
    small problem (the paper's Table of condition estimates shows the same order of
    agreement); with IC(0) the errors are rich in the bottom eigenvectors of M^-1 A instead
    and only the bracket holds."""
    p = wl.small_3d(6, seed=4, dt=np.inf)
    ev = np.linalg.eigvalsh(p.scipy().toarray())
    v0 = np.random.default_rng(13).standard_normal(p.n)
    est = oracle.pcg_cond_estimate(p, p.source, v0, m=12, tol=1e-10, maxit=2000, precond=precond)
    assert est["lmax"] <= ev[-1] * (1 + 1e-12) and est["lmin"] >= ev[0] * (1 - 1e-10)
    assert est["kappa"] <= ev[-1] / ev[0] * (1 + 1e-10)
    if not precond:
        assert est["lmax"] == pytest.approx(ev[-1], rel=1e-6)
        assert est["lmin"] == pytest.approx(ev[0], rel=0.1)
    lam_k, _ = oracle.power_method(p, v0, est["iters"])
    assert lam_k == est["lmax"]


def test_build_w_basis_and_ritz_values():
    """Q is orthonormal, spans the error vectors (Eq. ek/ekd), E is W^T A W, and the Ritz
    values of unpreconditioned sampling lie inside the spectrum with the smallest one close
    to lambda_min (Section 5.2, 'Verification of Ritz vector')."""
    p = wl.small_3d(6, seed=4, dt=np.inf)
    A = p.scipy()
    out = oracle.System(p, None).solve(p.source, tol=1e-10, sample_m=12, maxit=2000)
    aux, info = oracle.build_w(p, out["x"], out["samples"], out["sample_iter"])
    W = aux.W
    np.testing.assert_allclose(W.T @ W, np.eye(W.shape[1]), atol=1e-12)
    Eh = out["x"][:, None] - out["samples"]
    proj = Eh - W @ (W.T @ Eh)
    assert np.linalg.norm(proj) <= 1e-6 * np.linalg.norm(Eh)
    np.testing.assert_allclose(aux.E, W.T @ (A @ W), rtol=1e-12, atol=1e-9)
    ev = np.linalg.eigvalsh(A.toarray())
    assert ev[0] * (1 - 1e-10) <= aux.ritz.min() and aux.ritz.max() <= ev[-1] * (1 + 1e-10)
    assert aux.ritz.min() == pytest.approx(ev[0], rel=0.1)
    # the Ritz vector of the smallest Ritz value is close to the smallest eigenvector
    w, V = np.linalg.eigh(A.toarray())
    rv, T = np.linalg.eigh(aux.E)
    v1 = W @ T[:, 0]
    assert abs(v1 @ V[:, 0]) > 0.9


def test_build_w_rank_deficient_samples():
    """Duplicated sample columns: the kept rank drops and the span is unchanged."""
    p = wl.small_3d(5, seed=4)
    out = oracle.System(p, oracle.IC0(p)).solve(p.source, tol=1e-10, sample_m=6)
    s = out["samples"].copy()
    s[:, 5] = s[:, 4]
    aux, info = oracle.build_w(p, out["x"], s, out["sample_iter"])
    assert info["mbar"] == 5 and aux.m == 5


def test_theta_filter_keeps_small_ritz():
    p = wl.small_3d(6, seed=4, dt=np.inf)
    out = oracle.System(p, None).solve(p.source, tol=1e-10, sample_m=12, maxit=2000)
    aux_all, info = oracle.build_w(p, out["x"], out["samples"], out["sample_iter"])
    theta = np.sort(info["ritz"])[3] * 1.0000001
    aux, info2 = oracle.build_w(p, out["x"], out["samples"], out["sample_iter"], theta=theta)
    assert aux.m == 4
    np.testing.assert_allclose(np.diag(aux.E), np.sort(info["ritz"])[:4], rtol=1e-10)


# ---------------------------------------------------------------- sequence behaviour

@pytest.fixture(scope="module")
def c1_sequences():
    p = wl.config_c1()
    return p, {mode: oracle.run_sequence(p, 5, mode, 8) for mode in (0, 1, 2)}


def test_sequence_iteration_cut(c1_sequences):
    """W from sampled errors cuts iterations on systems 2..5 (Section 5.2); SC and deflation
    behave alike (Section 5.2, 'the convergence properties of two solvers were almost the
    same')."""
    p, seq = c1_sequences
    it = {m: [r["iters"] for r in seq[m][0]] for m in seq}
    for t in range(1, 5):
        assert it[1][t] < 0.7 * it[0][t] and it[2][t] < 0.7 * it[0][t]
        assert abs(it[1][t] - it[2][t]) <= 0.15 * it[0][t]


def test_sequence_true_residuals(c1_sequences):
    """The deflated residual equals the true residual of the corrected x (Eq. x1/x2)."""
    p, seq = c1_sequences
    A = p.scipy()
    x_prev = np.zeros(p.n)
    for r in seq[1][0]:
        b = x_prev / p.dt + p.source
        true = np.linalg.norm(b - A @ r["x"]) / np.linalg.norm(b)
        assert true <= 1.05e-8
        assert true == pytest.approx(r["relres"], rel=1e-3, abs=1e-12)
        x_prev = r["x"]


def test_modes_agree_on_solution(c1_sequences):
    p, seq = c1_sequences
    for t in range(5):
        x0 = seq[0][0][t]["x"]
        for m in (1, 2):
            assert np.linalg.norm(seq[m][0][t]["x"] - x0) <= 1e-6 * np.linalg.norm(x0)


# ---- sampling method B (Section 4.2: the relative residual levels)

def _levels_first_reached(res, tol, m, stop_iter):
    """Per level s = 1..m, the first iteration i (1 <= i < stop_iter) with
    ||r_i||/||b|| <= tol^(s/(m+1)) -- read off the residual history, squared as the
    method compares."""
    out = []
    for s in range(1, m + 1):
        lev2 = (tol * tol) ** (s / (m + 1))
        hit = [i for i in range(1, stop_iter) if res[i] * res[i] <= lev2]
        if hit:
            out.append(hit[0])
    return sorted(set(out))


@pytest.mark.parametrize("name", ["c1", "small3d"])
def test_sampling_b_samples_first_crossings(name):
    """Method B stores exactly the iterates at which a new residual level is first reached
    (an iteration reaching several levels once), none at the stopping iteration."""
    p = wl.config_c1() if name == "c1" else wl.small_3d(9, seed=11)
    b = p.source if p.source is not None else wl.random_rhs(p.n, 4)
    m, tol = 8, 1e-8
    out = oracle.System(p, oracle.IC0(p)).solve(b, tol=tol, sample_m=m, sample_method=1)
    si = out["sample_iter"]
    filled = sorted(int(v) for v in si if v > 0)
    assert filled == _levels_first_reached(out["res"], tol, m, out["iters"])
    assert list(si[:len(filled)]) == filled  # slots fill in order
    assert np.all(si[len(filled):] == 0)


def test_sampling_b_columns_are_the_iterates():
    """Each stored column is the iterate after that many iterations (a rerun with maxit set
    to the sample's iteration, same arithmetic)."""
    p = wl.config_c1()
    sysm = oracle.System(p, oracle.IC0(p))
    out = sysm.solve(p.source, tol=1e-8, sample_m=6, sample_method=1)
    for k, it in enumerate(out["sample_iter"]):
        if it <= 0:
            continue
        xk = sysm.solve(p.source, tol=1e-300, maxit=int(it), history=False)["x"]
        assert np.array_equal(out["samples"][:, k], xk), k

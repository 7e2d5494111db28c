"""The seeded generators against the configurations they stand for (CPU only): sizes, colour
counts, coefficient ranges, and the structure the method relies on (symmetric, weakly
diagonally dominant with a strictly dominant row, no coupling inside a colour)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as wl


def _check_structure(p, dominance=True):
    A = p.scipy()
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    assert p.colour_ptr[0] == 0 and p.colour_ptr[-1] == p.n
    colour = np.repeat(np.arange(p.ncolours), np.diff(p.colour_ptr))
    C = A.tocoo()
    off = C.row != C.col
    assert not np.any(colour[C.row[off]] == colour[C.col[off]]), "a colour couples two of its rows"
    if dominance:
        d = A.diagonal()
        offsum = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
        assert np.all(d > 0) and np.all(d >= offsum * (1 - 1e-12))
        assert np.any(d > offsum * (1 + 1e-9))


def test_c1_64x64_red_black_four_square_inclusions():
    p = wl.config_c1()
    assert p.n == 64 * 64 and p.nnz == 5 * 4096 - 4 * 64 == 20224
    assert p.ncolours == 2
    assert np.count_nonzero(p.coef == 1e3) == 4 * 36 and set(np.unique(p.coef)) == {1.0, 1e3}
    assert p.source is not None and p.source.min() >= 0.0 and p.source.max() < 1.0
    _check_structure(p)


def test_c2_128cube_eight_colours_sixteen_balls():
    p = wl.config_c2()
    n = 128 ** 3
    assert p.n == n == 2_097_152 and p.nnz == 7 * n - 6 * 128 ** 2 == 14_581_760
    assert p.ncolours == 8
    assert set(np.unique(p.coef)) == {1.0, 1e5}
    # sixteen separate balls of radius 4..8 cells: their volume lies between 16 (4/3 pi 4^3)
    # and 16 (4/3 pi 8^3) up to the rasterisation of the surface
    vol = np.count_nonzero(p.coef == 1e5)
    assert 16 * 4 / 3 * np.pi * 3.5 ** 3 <= vol <= 16 * 4 / 3 * np.pi * 8.5 ** 3
    assert p.dt == 1e-3
    _check_structure(p)


@pytest.mark.parametrize("N", [4, 7])
def test_fe27_nnz_formula_and_structure(N):
    """Q1 elements on (N+1)^3 cells with Dirichlet nodes eliminated: (3N - 2)^3 entries, and
    the 8-colouring (i%2 + 2 j%2 + 4 k%2) has no coupling inside a colour for 27 points."""
    p = wl.config_c3(N=N)
    assert p.n == N ** 3 and p.nnz == (3 * N - 2) ** 3
    assert p.ncolours == 8
    _check_structure(p, dominance=False)  # FE stiffness with 1e-3 anisotropy is not an M-matrix
    ev = np.linalg.eigvalsh(p.scipy().toarray())
    assert ev[0] > 0


def test_c5_recipe_is_c2_at_twice_the_resolution():
    """C5 keeps C2's operator and colouring with 64 balls of 1e6; at a reduced size the same
    recipe gives the same sizes and structure."""
    p = wl.config_c5(N=48, count=4, rmin=3.0, rmax=6.0)
    assert p.n == 48 ** 3 and p.nnz == 7 * p.n - 6 * 48 ** 2 and p.ncolours == 8
    assert set(np.unique(p.coef)) == {1.0, 1e6}
    _check_structure(p)


def test_generators_are_seeded():
    a, b = wl.config_c1(), wl.config_c1()
    assert np.array_equal(a.val, b.val) and np.array_equal(a.source, b.source)
    c = wl.config_c1(seed=wl.SEED_BASE + 99)
    assert not np.array_equal(a.source, c.source)


def test_reorder_is_a_symmetric_permutation():
    p = wl.small_3d(6, seed=3)
    q = wl.reorder(p, wl.wavefront_colours(p.shape))
    A = p.scipy()
    B = q.scipy()
    inv = np.empty(p.n, dtype=np.int64)
    inv[p.perm] = np.arange(p.n)
    Q = inv[q.perm]  # row of q -> row of p
    assert abs(B - A[Q][:, Q]).max() == 0
    assert np.array_equal(q.source, p.source[Q])
    _check_structure(q)
    assert sp.issparse(B)

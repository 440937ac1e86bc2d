"""Pins of the oracle's H-matrix for two point sets, A_{phi, Y1 x Y2} (Sec.
6.1: the paper's library builds the matrix of a kernel on sets Y1 and Y2).
Each set is ordered and clustered on its own; Alg. 1 runs from the pair of
roots with tau in Y1's tree and sigma in Y2's."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _kernel_matrix(P, Q, kernel, ell):
    D2 = ((P[:, None, :] - Q[None, :, :]) ** 2).sum(-1)
    if kernel == 0:
        return np.exp(-D2 / ell ** 2)
    s = np.sqrt(3 * D2) / ell
    return (1 + s) * np.exp(-s)


def test_rect_dense_matvec_matches_numpy(orc):
    P = inputs.uniform_points(250, 2, 3)
    Q = inputs.mixture_points(400, 2, 4)
    x = inputs.normal_vector(400, 5)
    for kern in (0, 1):
        want = _kernel_matrix(P, Q, kern, 0.15) @ x
        assert np.allclose(orc.dense_matvec_rect(P, Q, kern, 0.15, x), want, rtol=1e-13,
                           atol=1e-13)


def test_rect_same_set_is_the_square_build(orc):
    """With Y2 = Y1 every step takes the same operands as the square build:
    the same leaves, ranks and product, bit for bit."""
    pts = inputs.uniform_points(1500, 2, 7)
    x = inputs.normal_vector(1500, 8)
    S = orc.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-8)
    R = orc.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-8, cols=pts)
    assert np.array_equal(R.adm_leaves(), S.adm_leaves())
    assert np.array_equal(R.dense_leaves(), S.dense_leaves())
    assert np.array_equal(R.ranks()[0], S.ranks()[0])
    assert np.array_equal(R.col_perm(), S.perm())
    assert np.array_equal(R.matvec(x), S.matvec(x))


@pytest.mark.parametrize("n1,n2,leaf", [(700, 1100, 16), (300, 4000, 32), (2048, 64, 8),
                                        (1, 500, 8)])
def test_rect_leaves_tile_the_product_index_set(orc, n1, n2, leaf):
    """Every (i, j) of I1 x I2 lies in exactly one leaf; admissible leaves
    pass the test of Sec. 2.3; a dense leaf has a side of at most C_leaf."""
    P = inputs.uniform_points(n1, 2, 11)
    Q = inputs.halton_points(n2, 2)
    H = orc.HMatrix(P, 0, 0.2, leaf, 1.0, 1e-6, compress=False, cols=Q)
    lo, hi, bmin, bmax = H.tree()
    lo2, hi2, bmin2, bmax2 = H.col_tree()
    cover = np.zeros((n1, n2), np.int32)
    for t, s in H.adm_leaves():
        cover[lo[t]:hi[t], lo2[s]:hi2[s]] += 1
        dt = np.sum((bmax[t] - bmin[t]) ** 2)
        ds = np.sum((bmax2[s] - bmin2[s]) ** 2)
        g = np.maximum(0, bmin[t] - bmax2[s]) ** 2 + np.maximum(0, bmin2[s] - bmax[t]) ** 2
        assert min(dt, ds) <= g.sum() * (1 + 1e-12)
    for t, s in H.dense_leaves():
        cover[lo[t]:hi[t], lo2[s]:hi2[s]] += 1
        assert min(hi[t] - lo[t], hi2[s] - lo2[s]) <= leaf
    assert (cover == 1).all()


@pytest.mark.parametrize("kern", [0, 1, 2])
def test_rect_exact_cases(orc, kern):
    P = inputs.uniform_points(400, 3, 13)
    Q = inputs.uniform_points(650, 3, 14)
    x = inputs.normal_vector(650, 15)
    yb = orc.dense_matvec_rect(P, Q, kern, 0.3, x)
    H0 = orc.HMatrix(P, kern, 0.3, 16, 0.0, 1e-6, cols=Q)       # eta = 0: all dense
    assert H0.n_adm == 0
    assert _rel(H0.matvec(x), yb) <= 1e-13
    H1 = orc.HMatrix(P, kern, 0.3, 650, 1.0, 1e-6, cols=Q)      # C >= N1, N2: one block
    assert H1.n_dense == 1 and H1.n_adm == 0
    assert _rel(H1.matvec(x), yb) <= 1e-13


@pytest.mark.parametrize("kern,ell", [(0, 0.1), (1, 0.2), (2, 0.2)])
def test_rect_error_within_eps(orc, kern, ell):
    P = inputs.uniform_points(3000, 2, 17)
    Q = inputs.mixture_points(2000, 2, 18)
    x = inputs.normal_vector(2000, 19)
    H = orc.HMatrix(P, kern, ell, 32, 1.0, 1e-8, cols=Q)
    assert H.n_adm > 0
    e = _rel(H.matvec(x), orc.dense_matvec_rect(P, Q, kern, ell, x))
    assert e <= 1e-7, e


def test_rect_swapped_sets_are_transposes(orc):
    """A(Y2, Y1) = A(Y1, Y2)^T for a symmetric kernel, so z^T (H12 x) and
    x^T (H21 z) agree up to the approximation error."""
    P = inputs.uniform_points(1800, 2, 21)
    Q = inputs.halton_points(1200, 2)
    x = inputs.normal_vector(1200, 22)
    z = inputs.normal_vector(1800, 23)
    H12 = orc.HMatrix(P, 0, 0.15, 32, 1.0, 1e-8, cols=Q)
    H21 = orc.HMatrix(Q, 0, 0.15, 32, 1.0, 1e-8, cols=P)
    a, b = z @ H12.matvec(x), x @ H21.matvec(z)
    scale = np.linalg.norm(z) * np.linalg.norm(orc.dense_matvec_rect(P, Q, 0, 0.15, x))
    assert abs(a - b) <= 1e-7 * scale

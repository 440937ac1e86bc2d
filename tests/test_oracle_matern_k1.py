"""Pins of the oracle's Matern kernel of order 1 (Sec. 6.2: beta - d/2 = 1),
phi(r) = s K_1(s) with s = r / l, normalised to phi(0) = 1.

The oracle evaluates K_1 by its ascending series (x <= 2) and by the
trapezoidal rule on its integral representation (x > 2). These tests tie it
to an independent library (scipy's k1), to the closed forms of K_1 at small
and large argument, and to the brute-force product."""
import math

import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

K1 = 2
EULER = 0.5772156649015329


def _phi(orc, s, ell=1.0):
    a = np.array([0.0, 0.0, 0.0])
    b = np.array([s * ell, 0.0, 0.0])
    return orc.kernel_eval(K1, ell, a, b)


def test_k1_matches_scipy(orc):
    sp = pytest.importorskip("scipy.special")
    s = np.concatenate([np.logspace(-8, 2.5, 300), [1.999999, 2.0, 2.000001, 1e-300 ** 0.5]])
    got = np.array([_phi(orc, v) for v in s])
    want = s * sp.k1(s)
    rel = np.abs(got - want) / want
    assert rel.max() <= 2e-14, (s[rel.argmax()], rel.max())


def test_k1_small_argument_closed_form(orc):
    # s K_1(s) = 1 + (s^2/2)(ln(s/2) + gamma - 1/2) + O(s^4 ln s)
    for s in (1e-3, 1e-4, 1e-5):
        want = 1.0 + 0.5 * s * s * (math.log(0.5 * s) + EULER - 0.5)
        assert abs(_phi(orc, s) - want) <= 4 * s ** 4 * abs(math.log(s)) + 2e-16
    assert _phi(orc, 0.0) == 1.0


def test_k1_large_argument_asymptotic(orc):
    # Hankel's expansion for order 1 (mu = 4):
    # K_1(s) ~ sqrt(pi/(2s)) e^-s (1 + 3/(8s) - 15/(128s^2) + 315/(3072s^3) - ...)
    for s in (200.0, 400.0):
        series = 1 + 3 / (8 * s) - 15 / (128 * s * s) + 315 / (3072 * s ** 3)
        want = s * math.sqrt(math.pi / (2 * s)) * math.exp(-s) * series
        assert abs(_phi(orc, s) / want - 1) <= 0.2 / s ** 4


def test_k1_length_scale_and_symmetry(orc):
    a = np.array([0.1, 0.7])
    b = np.array([0.45, 0.2])
    r = float(np.linalg.norm(a - b))
    for ell in (0.05, 0.3, 1.0):
        v = orc.kernel_eval(K1, ell, a, b)
        assert v == orc.kernel_eval(K1, ell, b, a)
        assert v == pytest.approx(_phi(orc, r / ell), rel=1e-15)
    assert orc.kernel_eval(K1, 0.3, a, a) == 1.0


def test_k1_dense_matvec_matches_scipy_matrix(orc):
    sp = pytest.importorskip("scipy.special")
    pts = inputs.uniform_points(300, 3, 19)
    x = inputs.normal_vector(300, 4)
    r = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)) / 0.2
    with np.errstate(invalid="ignore"):
        A = np.where(r > 0, r * sp.k1(np.where(r > 0, r, 1.0)), 1.0)
    y = orc.dense_matvec(pts, K1, 0.2, 0.1, x)
    assert np.allclose(y, A @ x + 0.1 * x, rtol=1e-13, atol=1e-13)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("d", [2, 3])
def test_k1_hmatrix_eta0_is_exact(orc, d):
    pts = inputs.uniform_points(500, d, 23)
    x = inputs.normal_vector(500, 6)
    h = orc.HMatrix(pts, K1, 0.2, 16, 0.0, 1e-6)
    assert h.n_adm == 0
    assert _rel(h.matvec(x), orc.dense_matvec(pts, K1, 0.2, 0.0, x)) <= 1e-13


@pytest.mark.parametrize("d,ell", [(2, 1.0), (3, 0.2)])
def test_k1_hmatrix_error_within_eps(orc, d, ell):
    # Sec. 6.4's setting (eta = 1.5) with the eps-adaptive ACA: the product's
    # error against brute force is of the order of eps
    n = 2048
    pts = inputs.halton_points(n, d) if d == 2 else inputs.uniform_points(n, d, 31)
    x = inputs.normal_vector(n, 8)
    h = orc.HMatrix(pts, K1, ell, 32, 1.5, 1e-8)
    assert h.n_adm > 0
    e = _rel(h.matvec(x), orc.dense_matvec(pts, K1, ell, 0.0, x))
    assert e <= 1e-7, e


def test_k1_fixed_rank_converges_geometrically(orc):
    # Sec. 6.4: e_rel of the product decays exponentially in the fixed ACA
    # rank k, for the Matern kernel as for the Gaussian (Halton points,
    # unscaled kernel, eta = 1.5)
    pts = inputs.halton_points(2048, 2)
    x = inputs.normal_vector(2048, 5)
    yb = orc.dense_matvec(pts, K1, 1.0, 0.0, x)
    errs = []
    for k in (2, 4, 8, 12):
        h = orc.HMatrix(pts, K1, 1.0, 32, 1.5, 0.0, k_cap=k)
        errs.append(_rel(h.matvec(x), yb))
    assert all(b < 0.2 * a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6, errs

"""A_{phi, Y1 x Y2} for two point sets (Sec. 6.1) on the GPU through the C-ABI
(hm_build_rect) against the CPU oracle: each set's permutation and the leaf
lists bit-exact, FP64 product within 1e-10, mixed precision within 1e-5, the
on-the-fly product equal to the stored one, several vectors, device tensors,
and the arguments a rectangular matrix refuses."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5

CASES = {
    # rows, cols (kind, n, seed), d, kernel, ell, leaf, eta, eps
    "gauss2d": (("u", 3000, 31), ("m", 2000, 32), 2, 0, 0.1, 32, 1.0, 1e-8),
    "matern3d": (("u", 2500, 33), ("u", 4000, 34), 3, 1, 0.2, 64, 1.0, 1e-6),
    "k1_2d": (("h", 2000, 0), ("u", 1500, 35), 2, 2, 0.2, 32, 1.0, 1e-8),
    "unbalanced": (("u", 300, 36), ("m", 5000, 37), 2, 0, 0.15, 32, 1.0, 1e-8),
    "one_row": (("u", 1, 38), ("u", 700, 39), 2, 1, 0.3, 16, 1.0, 1e-8),
    "fixed_rank": (("h", 4096, 0), ("u", 3000, 40), 2, 0, 1.0, 128, 1.5, 0.0),
}


@pytest.fixture(scope="module")
def hm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm as H
    build.build()
    H.lib()
    return H


def _pts(kind, n, seed, d):
    if kind == "h":
        return inputs.halton_points(n, d)
    return inputs.uniform_points(n, d, seed) if kind == "u" else inputs.mixture_points(n, d, seed)


_ORACLE = {}


def _case(orc, name):
    if name not in _ORACLE:
        r, c, d, kern, ell, leaf, eta, eps = CASES[name]
        P, Q = _pts(*r, d), _pts(*c, d)
        k_cap = 16 if eps <= 0 else 64
        O = orc.HMatrix(P, kern, ell, leaf, eta, eps, k_cap=k_cap, cols=Q)
        x = inputs.normal_vector(Q.shape[0], inputs.X_SEED)
        _ORACLE[name] = (P, Q, x, O, O.matvec(x), k_cap)
    return _ORACLE[name]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name", list(CASES))
def test_structure_and_fp64_product(hm, orc, name):
    r, c, d, kern, ell, leaf, eta, eps = CASES[name]
    P, Q, x, O, yo, k_cap = _case(orc, name)
    H = hm.HMatrix(P, kern, ell, leaf, eta, eps, k_cap=k_cap, cols=Q)
    s = H.structure()
    n1 = P.shape[0]
    assert np.array_equal(s["perm"][:n1], O.perm())
    assert np.array_equal(s["perm"][n1:], O.col_perm())
    assert np.array_equal(s["adm"], O.adm_leaves())
    assert np.array_equal(s["dense"], O.dense_leaves())
    if eps > 0:
        oranks, _ = O.ranks()
        assert int((s["ranks"] != oranks).sum()) <= max(1, len(oranks) // 1000)
    y = H.matvec(x)
    assert y.shape == (n1,)
    e = rel(y, yo)
    assert e <= FP64_TOL, e


@pytest.mark.parametrize("name", ["gauss2d", "matern3d", "k1_2d", "unbalanced"])
def test_mixed_precision_product(hm, orc, name):
    r, c, d, kern, ell, leaf, eta, eps = CASES[name]
    P, Q, x, O, yo, k_cap = _case(orc, name)
    H = hm.HMatrix(P, kern, ell, leaf, eta, eps, k_cap=k_cap, cols=Q, precision=hm.PREC_MIXED)
    e = rel(H.matvec(x), yo)
    assert e <= MIXED_TOL, e


def test_same_set_matches_square_handle(hm, orc):
    P = inputs.uniform_points(4000, 2, 41)
    x = inputs.normal_vector(4000, 42)
    S = hm.HMatrix(P, 0, 0.1, 32, 1.0, 1e-8)
    R = hm.HMatrix(P, 0, 0.1, 32, 1.0, 1e-8, cols=P)
    assert np.array_equal(R.structure()["adm"], S.structure()["adm"])
    assert rel(R.matvec(x), S.matvec(x)) <= 1e-14


@pytest.mark.parametrize("name", ["gauss2d", "unbalanced"])
def test_on_the_fly_matches_stored(hm, orc, name):
    r, c, d, kern, ell, leaf, eta, eps = CASES[name]
    P, Q, x, O, yo, k_cap = _case(orc, name)
    S = hm.HMatrix(P, kern, ell, leaf, eta, eps, k_cap=k_cap, cols=Q)
    F = hm.HMatrix(P, kern, ell, leaf, eta, eps, k_cap=k_cap, cols=Q, on_the_fly=True)
    yf = F.matvec(x)
    assert rel(yf, S.matvec(x)) <= 1e-13
    assert rel(yf, yo) <= FP64_TOL


def test_several_vectors_accumulate_and_device_tensors(hm, orc):
    import torch
    P, Q, x, O, yo, k_cap = _case(orc, "gauss2d")
    r, c, d, kern, ell, leaf, eta, eps = CASES["gauss2d"]
    H = hm.HMatrix(P, kern, ell, leaf, eta, eps, cols=Q)
    X = np.stack([x, 2.0 * x, inputs.normal_vector(Q.shape[0], 43)])
    Y = H.matvec(X)
    assert Y.shape == (3, P.shape[0])
    assert rel(Y[0], yo) <= FP64_TOL
    assert np.allclose(Y[1], 2.0 * Y[0], rtol=1e-14, atol=0)
    assert rel(Y[2], O.matvec(X[2])) <= FP64_TOL
    yt = H.matvec(torch.from_numpy(x).cuda())
    assert rel(yt.cpu().numpy(), yo) <= FP64_TOL
    A = hm.HMatrix(P, kern, ell, leaf, eta, eps, cols=Q, accumulate=True)
    y0 = np.ones(P.shape[0])
    y1 = A.matvec(x, y0.copy())
    assert rel(y1 - y0, yo) <= FP64_TOL


def test_rectangular_refusals(hm, orc):
    P = inputs.uniform_points(500, 2, 44)
    Q = inputs.uniform_points(600, 2, 45)
    with pytest.raises(hm.HMError) as e:
        hm.HMatrix(P, 0, 0.1, 32, 1.0, 1e-6, sigma2=0.1, cols=Q)
    assert e.value.code == -1
    with pytest.raises(hm.HMError) as e:
        hm.HMatrix(P, 0, 0.1, 32, 1.0, 1e-6, cols=Q, symmetric=True)
    assert e.value.code == -6
    with pytest.raises(hm.HMError):
        hm.HMatrix(P, 0, 0.1, 32, 1.0, 1e-6, cols=inputs.uniform_points(600, 3, 45))
    H = hm.HMatrix(P, 0, 0.1, 32, 1.0, 1e-6, cols=Q)
    with pytest.raises(hm.HMError) as e:
        H.cg(np.ones(500))
    assert e.value.code == -1


def test_mixed_floor_keeps_ranks_below_the_cap(hm, orc):
    """Mixed precision for two sets: the floor of the ACA tests (with the
    dense leaves' sum of squares as its bound of ||A||_F^2) stops blocks whose
    entries lie near float underflow before they fit rounding noise up to the
    rank cap, and the product stays within 1e-5 of the oracle."""
    P = inputs.mixture_points(1 << 15, 2, 51)
    Q = inputs.halton_points(1 << 14, 2)
    x = inputs.normal_vector(1 << 14, 52)
    O = orc.HMatrix(P, 0, 0.1, 64, 1.0, 1e-6, cols=Q)
    H = hm.HMatrix(P, 0, 0.1, 64, 1.0, 1e-6, cols=Q, precision=hm.PREC_MIXED)
    st = H.stats()
    assert st["rank_cap_hits"] == 0, st["rank_cap_hits"]
    assert st["max_rank"] <= int(O.ranks()[0].max()) + 8
    e = rel(H.matvec(x), O.matvec(x))
    assert e <= MIXED_TOL, e

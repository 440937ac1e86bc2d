"""The Matern kernel of order 1 (Sec. 6.2, beta - d/2 = 1; phi = s K_1(s),
s = r / l) on the GPU through the C-ABI against the CPU oracle: structure
bit-exact, FP64 product within 1e-10, mixed precision within 1e-5, the
on-the-fly product equal to the stored one, and entries evaluated in both
branches of the device's K_1 (s <= 2 and s > 2)."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5
K1 = 2

CASES = {
    # n, d, kind, ell, leaf, eta, adm_max, eps
    "u2d": (2048, 2, "u", 0.1, 32, 1.0, True, 1e-8),     # s up to 14: both branches
    "u3d": (3000, 3, "u", 0.3, 32, 1.0, False, 1e-6),
    "mix2d": (3000, 2, "m", 0.1, 64, 1.0, False, 1e-6),  # clipped mixture: duplicates
    # the paper's setting scaled down: Halton points, unscaled kernel,
    # eta = 1.5, fixed rank 16 (Sec. 6.7)
    "paper": (8192, 2, "h", 1.0, 128, 1.5, False, 0.0),
    "eta0": (1000, 2, "u", 0.2, 8, 0.0, False, 1e-6),    # every block dense
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


_ORACLE = {}


def _case(orc, name):
    """Points, x, the oracle's H-matrix and its product, built once per case."""
    if name not in _ORACLE:
        n, d, kind, ell, leaf, eta, adm_max, eps = CASES[name]
        if kind == "h":
            pts = inputs.halton_points(n, d)
        elif kind == "u":
            pts = inputs.uniform_points(n, d, 11)
        else:
            pts = inputs.mixture_points(n, d, 11)
        x = inputs.normal_vector(n, inputs.X_SEED)
        k_cap = 16 if eps <= 0 else 64
        O = orc.HMatrix(pts, K1, ell, leaf, eta, eps, adm_max=adm_max, k_cap=k_cap)
        _ORACLE[name] = (pts, x, O, O.matvec(x), k_cap)
    return _ORACLE[name]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name", list(CASES))
def test_structure_and_fp64_product(hm, orc, name):
    n, d, kind, ell, leaf, eta, adm_max, eps = CASES[name]
    pts, x, O, yo, k_cap = _case(orc, name)
    H = hm.HMatrix(pts, K1, ell, leaf, eta, eps, adm_max=adm_max, k_cap=k_cap)
    s = H.structure()
    assert np.array_equal(s["perm"], O.perm())
    assert np.array_equal(s["adm"], O.adm_leaves())
    assert np.array_equal(s["dense"], O.dense_leaves())
    if eps > 0:
        oranks, _ = O.ranks()
        assert int((s["ranks"] != oranks).sum()) <= max(1, len(oranks) // 1000)
    e = rel(H.matvec(x), yo)
    assert e <= (1e-13 if eta == 0 else FP64_TOL), e


@pytest.mark.parametrize("near", ["bf16x2", "fp32"])
@pytest.mark.parametrize("name", ["u2d", "u3d", "mix2d", "paper"])
def test_mixed_precision_product(hm, orc, name, near):
    n, d, kind, ell, leaf, eta, adm_max, eps = CASES[name]
    pts, x, O, yo, k_cap = _case(orc, name)
    fmt = {"bf16x2": hm.NEAR_BF16X2, "fp32": hm.NEAR_FP32}[near]
    H = hm.HMatrix(pts, K1, ell, leaf, eta, eps, adm_max=adm_max, k_cap=k_cap,
                   precision=hm.PREC_MIXED, near_format=fmt)
    e = rel(H.matvec(x), yo)
    assert e <= MIXED_TOL, e


def test_dense_entries_in_float(hm, orc):
    """eta = 0: the product is the dense matrix, so the float kernel's entries
    (both branches of K_1) decide the error alone."""
    n, d, kind, ell, leaf, eta, adm_max, eps = CASES["eta0"]
    pts, x, O, yo, k_cap = _case(orc, "eta0")
    H = hm.HMatrix(pts, K1, ell, leaf, eta, eps, precision=hm.PREC_MIXED,
                   near_format=hm.NEAR_FP32)
    e = rel(H.matvec(x), yo)
    assert e <= 2e-6, e


@pytest.mark.parametrize("name", ["u2d", "paper"])
def test_on_the_fly_matches_stored(hm, orc, name):
    n, d, kind, ell, leaf, eta, adm_max, eps = CASES[name]
    pts, x, O, yo, k_cap = _case(orc, name)
    S = hm.HMatrix(pts, K1, ell, leaf, eta, eps, adm_max=adm_max, k_cap=k_cap)
    F = hm.HMatrix(pts, K1, ell, leaf, eta, eps, adm_max=adm_max, k_cap=k_cap, on_the_fly=True)
    yf = F.matvec(x)
    assert rel(yf, S.matvec(x)) <= 1e-13
    assert rel(yf, yo) <= FP64_TOL
    M = hm.HMatrix(pts, K1, ell, leaf, eta, eps, adm_max=adm_max, k_cap=k_cap, on_the_fly=True,
                   precision=hm.PREC_MIXED)
    assert rel(M.matvec(x), yo) <= MIXED_TOL

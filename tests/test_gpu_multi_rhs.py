"""Product with several right-hand sides in one call (Alg. 3 applied to the
columns of X): every column matches the oracle within the mixed-precision
bound, and the result of a column does not depend on the columns it is
grouped with (group widths 8 and 16, padding, several groups per call)."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5
FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def hm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm as H
    build.build()
    H.lib()
    return H


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _pts(n, d, kind, seed):
    if kind == "m":
        return inputs.mixture_points(n, d, seed)
    return inputs.uniform_points(n, d, seed)


def _rhs(n, k, seed0=500):
    return np.stack([inputs.normal_vector(n, seed0 + r) for r in range(k)])


@pytest.mark.parametrize("near", ["bf16x2", "fp32", "fp64"])
def test_columns_match_oracle_and_single_product(hm, orc, near):
    fmt = {"bf16x2": hm.NEAR_BF16X2, "fp32": hm.NEAR_FP32, "fp64": hm.NEAR_FP64}[near]
    n = 20000
    pts = _pts(n, 2, "m", 21)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, sigma2=0.01, precision=hm.PREC_MIXED,
                   near_format=fmt)
    O = orc.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, sigma2=0.01)
    X = _rhs(n, 12)
    Y = H.matvec(X)
    assert Y.shape == X.shape
    for r in range(12):
        assert rel(Y[r], O.matvec(X[r])) <= MIXED_TOL, r
        # the one-vector product sums in another order: both are compensated
        assert rel(Y[r], H.matvec(X[r])) <= 1e-6, r


def test_grouping_does_not_change_a_column(hm):
    n = 12345                                       # ragged last tile
    pts = _pts(n, 2, "u", 31)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, sigma2=0.01, precision=hm.PREC_MIXED)
    X = _rhs(n, 20)
    Y20 = H.matvec(X)                               # groups of 16 and 4 (width 8)
    Y12 = H.matvec(X[:12])                          # one group of width 16
    Y5 = H.matvec(X[:5])                            # width 8, three padding columns
    Y2 = H.matvec(X[3:5])                           # the same columns at other places
    assert np.array_equal(Y20[:12], Y12)
    assert np.array_equal(Y12[:5], Y5)
    assert np.array_equal(Y5[3:5], Y2)
    assert np.array_equal(Y20[16:], H.matvec(X[16:]))
    # repeated calls give the same bits
    assert np.array_equal(H.matvec(X[:12]), Y12)


def test_device_buffers_accumulate_and_3d(hm, orc):
    import torch
    n = 9000
    pts = _pts(n, 3, "u", 41)
    H = hm.HMatrix(pts, 1, 0.2, 64, 1.0, 1e-6, precision=hm.PREC_MIXED)
    X = _rhs(n, 9)
    Yh = H.matvec(X)
    Yd = H.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.array_equal(Yh, Yd)
    O = orc.HMatrix(pts, 1, 0.2, 64, 1.0, 1e-6)
    assert rel(Yh[8], O.matvec(X[8])) <= MIXED_TOL
    Ha = hm.HMatrix(pts, 1, 0.2, 64, 1.0, 1e-6, precision=hm.PREC_MIXED, accumulate=True)
    Y = np.ones_like(X)
    Ha.matvec(X, Y)
    assert np.array_equal(Y, Yh + 1.0)


@pytest.mark.parametrize("prec,leaf", [(0, 64), (1, 128)])
def test_unfused_plans_loop_the_single_product(hm, prec, leaf):
    """FP64 plans and slices of more than 64 rows run one product per vector."""
    n = 8000
    pts = _pts(n, 2, "m", 51)
    H = hm.HMatrix(pts, 0, 0.1, leaf, 1.0, 1e-6, precision=prec)
    X = _rhs(n, 3)
    Y = H.matvec(X)
    for r in range(3):
        assert np.array_equal(Y[r], H.matvec(X[r]))

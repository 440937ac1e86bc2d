"""Launch shapes of the batched ACA (Alg. 2, Sec. 5.4.1) against the oracle.

Every shape (the cluster kernels of the first design, the default team
kernels, the alternative team shapes) must give the same approximation: the
FP64 product within 1e-10 of the oracle's, mixed precision within 1e-5, the
ranks within a few blocks of each other. The workloads span the size classes
up to blocks of several thousand rows and, with a tight eps, reservations in
every rank bucket (ranks above 16 and 32). The iteration-limit test hook makes
the ACA loops give up, which must come back as HM_ETIMEOUT without a fault,
and a build afterwards must work again.
"""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def hm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm as H
    build.build()
    H.lib()
    yield H
    H.set_aca_shape(-1, -1)
    H.set_test_hook(H.HOOK_ACA_STEP_LIMIT, 0)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    # n, d, points, kernel, ell, leaf, eta, eps
    (1 << 15, 2, "m", 0, 0.1, 64, 1.0, 1e-6),     # the benchmark's mixture, smaller
    (8000, 3, "u", 1, 0.2, 32, 1.0, 1e-9),        # ranks above 32 (bucket 64)
    (12000, 2, "u", 2, 0.5, 48, 1.5, 1e-8),       # Matern of order 1
]


@pytest.mark.parametrize("case", CASES)
def test_every_aca_shape_matches_oracle_fp64(hm, orc, case):
    n, d, kind, kern, ell, leaf, eta, eps = case
    pts = inputs.uniform_points(n, d, 31) if kind == "u" else inputs.mixture_points(n, d, 31)
    x = inputs.normal_vector(n, inputs.X_SEED)
    O = orc.HMatrix(pts, kern, ell, leaf, eta, eps)
    yo = O.matvec(x)
    ro = O.ranks()[0]
    assert ro.max() > 16
    for shape in (0, 1, 2):
        hm.set_aca_shape(-1, shape)
        H = hm.HMatrix(pts, kern, ell, leaf, eta, eps)
        y = H.matvec(x)
        r = H.structure()["ranks"]
        H.free()
        assert rel(y, yo) <= FP64_TOL, (shape, rel(y, yo))
        # ranks agree except where a stopping test sits at a rounding boundary
        assert np.mean(r != ro) <= 2e-3, (shape, np.mean(r != ro))
    hm.set_aca_shape(-1, -1)


@pytest.mark.parametrize("sym", [False, True])
def test_every_aca_shape_mixed(hm, orc, sym):
    n = 1 << 15
    w = inputs.WORKLOADS["mix2d_n1m"]
    pts = inputs.workload_points("mix2d_n1m", n)
    x = inputs.normal_vector(n, inputs.X_SEED)
    O = orc.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], symmetric=sym)
    yo = O.matvec(x)
    ys = []
    for shape in (0, 1, 2):
        hm.set_aca_shape(-1, shape)
        H = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                       precision=hm.PREC_MIXED, symmetric=sym)
        ys.append(H.matvec(x))
        H.free()
        assert rel(ys[-1], yo) <= MIXED_TOL, (shape, rel(ys[-1], yo))
    hm.set_aca_shape(-1, -1)


def test_single_class_shape_override(hm, orc):
    # one class on the cluster kernels, the rest on the team kernels
    n = 1 << 15
    pts = inputs.mixture_points(n, 2, 5)
    x = inputs.normal_vector(n, inputs.X_SEED)
    O = orc.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6)
    yo = O.matvec(x)
    for cls in (0, 3, 5):
        hm.set_aca_shape(-1, -1)
        hm.set_aca_shape(cls, 0)
        H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6)
        assert rel(H.matvec(x), yo) <= FP64_TOL
        H.free()
    hm.set_aca_shape(-1, -1)
    with pytest.raises(hm.HMError):
        hm.set_aca_shape(12, 0)
    with pytest.raises(hm.HMError):
        hm.set_aca_shape(0, 3)


@pytest.mark.parametrize("shape", [0, 1])
def test_aca_step_limit_gives_timeout(hm, shape):
    # a limit of one iteration per block: every block with rank >= 2 stops at
    # its limit; the build reports HM_ETIMEOUT and no kernel faults
    n = 1 << 14
    pts = inputs.mixture_points(n, 2, 7)
    hm.set_aca_shape(-1, shape)
    hm.set_test_hook(hm.HOOK_ACA_STEP_LIMIT, 1)
    try:
        with pytest.raises(hm.HMError) as ei:
            hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6)
        assert ei.value.code == hm.ETIMEOUT
    finally:
        hm.set_test_hook(hm.HOOK_ACA_STEP_LIMIT, 0)
        hm.set_aca_shape(-1, -1)
    # the context is still usable
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6)
    y = H.matvec(inputs.normal_vector(n, 1))
    H.free()
    assert np.isfinite(y).all()
    with pytest.raises(hm.HMError):
        hm.set_test_hook(99, 1)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_shape_tuner_picks_a_shape_per_class(hm, orc, prec):
    n = 1 << 15
    pts = inputs.mixture_points(n, 2, 33)
    x = inputs.normal_vector(n, inputs.X_SEED)
    p = hm.PREC_FP64 if prec == "fp64" else hm.PREC_MIXED
    try:
        shapes = hm.tune_aca_shapes(pts, 0, 0.1, 64, 1.0, 1e-6, reps=1, precision=p)
        assert len(shapes) == 12 and set(shapes) <= {-1, 0, 1, 2}
        # the classes that hold blocks at N = 2^15 (rows up to 2^13) got a shape
        assert all(s >= 0 for s in shapes[:6]), shapes
        H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=p)
        y = H.matvec(x)
        H.free()
    finally:
        hm.set_aca_shape(-1, -1)
    yo = orc.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6).matvec(x)
    assert rel(y, yo) <= (FP64_TOL if prec == "fp64" else MIXED_TOL)
    with pytest.raises(hm.HMError):
        hm.tune_aca_shapes(pts, 0, 0.1, 64, 1.0, 1e-6, on_the_fly=True)

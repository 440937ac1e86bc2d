"""Batch sizes of the batched ACA and of the product's gather (Sec. 5.4.1
bs_ACA, Sec. 5.4.2 bs_dense; hm_set_batch_limits): every block and every
gather item computes the same values whatever launch it runs in, so ranks and
products are bit-identical from one launch per block (or item) up to one
launch per size class (or one gather launch)."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm as H
    build.build()
    H.lib()
    yield H
    H.set_batch_limits(0, 0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_aca_batch_sizes_give_the_same_factors(hm, prec):
    n = 1 << 14
    pts = inputs.mixture_points(n, 2, 41)
    x = inputs.normal_vector(n, 7)
    p = hm.PREC_FP64 if prec == "fp64" else hm.PREC_MIXED
    ref = None
    for bs in (0, 1 << 20, 1 << 16, 1):
        hm.set_batch_limits(bs, 0)
        try:
            H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=p)
        finally:
            hm.set_batch_limits(0, 0)
        y = H.matvec(x)
        rk = H.structure()["ranks"]
        H.free()
        if ref is None:
            ref = (y, rk)
            continue
        assert np.array_equal(rk, ref[1]), bs
        assert np.array_equal(y, ref[0]), bs


@pytest.mark.parametrize("shape", [0, 4])
def test_gather_items_per_launch_give_the_same_product(hm, shape):
    n = 1 << 15
    pts = inputs.mixture_points(n, 2, 42)
    x = inputs.normal_vector(n, 8)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED, sigma2=0.01)
    hm.set_gather_shape(shape)
    try:
        ref = H.matvec(x)
        for items in (1, 7, 100, 1 << 20):
            hm.set_batch_limits(0, items)
            y = H.matvec(x)
            assert np.array_equal(y, ref), items
    finally:
        hm.set_batch_limits(0, 0)
        hm.set_gather_shape(-1)
    H.free()

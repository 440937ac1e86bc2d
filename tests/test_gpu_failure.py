"""Failure paths, made to happen on purpose without a GPU fault.

- A bounded wait runs out: the bulk-copy producer of the product's gather
  leaves one chunk out (a test hook), so its consumers' mbarrier wait has
  nothing to wait for; with a 2 ms bound they give up, the product reports
  HM_ETIMEOUT (a host-buffer product at once, a device-buffer product at
  hm_check_status), and the next product is correct again.
- An allocation fails: the n-th device allocation from now is made to fail;
  the build returns HM_ENOMEM with no handle, and the library holds no more
  device memory afterwards than before.
- A level of the block-tree traversal does not fit its bound: with the
  first bound forced down to min(4^l, 2^l) pairs the traversal overflows on
  the device, the host runs it again with doubled bounds, and the leaf lists
  are those of a traversal that fitted at once; allowed a single traversal,
  the build returns HM_EOVERFLOW instead and holds no device memory after.
The ACA iteration-limit hook is covered in test_gpu_aca_shapes.py.
"""
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
    for hook in (H.HOOK_WAIT_LIMIT_NS, H.HOOK_GATHER_WITHHOLD, H.HOOK_FAIL_ALLOC,
                 H.HOOK_TRAVERSAL_KAPPA, H.HOOK_TRAVERSAL_TRIES):
        H.set_test_hook(hook, 0)
    H.set_gather_shape(-1)


def _mixed(hm, n=1 << 15, seed=21):
    pts = inputs.mixture_points(n, 2, seed)
    return pts, hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED)


@pytest.mark.parametrize("nrhs", [1, 4])
def test_withheld_chunk_times_out_and_recovers(hm, nrhs):
    import torch
    pts, H = _mixed(hm)
    n = pts.shape[0]
    hm.set_gather_shape(3)                 # the bulk-copy gather
    x = inputs.normal_vector(n, 5, nrhs=nrhs) if nrhs > 1 else inputs.normal_vector(n, 5)
    ref = H.matvec(x)
    hm.set_test_hook(hm.HOOK_WAIT_LIMIT_NS, 2_000_000)
    hm.set_test_hook(hm.HOOK_GATHER_WITHHOLD, 1 + 1)   # chunk 1 of every work item
    try:
        with pytest.raises(hm.HMError) as ei:
            H.matvec(x)                    # host buffers: checked before return
        assert ei.value.code == hm.ETIMEOUT
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        H.matvec(xd)                       # device buffers: reported on request
        with pytest.raises(hm.HMError) as ei:
            H.check_status()
        assert ei.value.code == hm.ETIMEOUT
    finally:
        hm.set_test_hook(hm.HOOK_GATHER_WITHHOLD, 0)
        hm.set_test_hook(hm.HOOK_WAIT_LIMIT_NS, 0)
    H.check_status()                       # cleared by the check
    y = H.matvec(x)
    assert np.array_equal(y, ref)
    H.free()
    hm.set_gather_shape(-1)


def test_short_wait_bound_alone_does_not_fail(hm):
    # every wait bounded at 50 ms: a product whose copies all arrive is
    # unaffected
    pts, H = _mixed(hm, seed=22)
    x = inputs.normal_vector(pts.shape[0], 6)
    hm.set_gather_shape(4)
    ref = H.matvec(x)
    hm.set_test_hook(hm.HOOK_WAIT_LIMIT_NS, 50_000_000)
    try:
        y = H.matvec(x)
    finally:
        hm.set_test_hook(hm.HOOK_WAIT_LIMIT_NS, 0)
        hm.set_gather_shape(-1)
    assert np.array_equal(y, ref)
    H.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_injected_allocation_failure(hm, prec):
    import torch
    n = 1 << 14
    pts = inputs.mixture_points(n, 2, 23)
    p = hm.PREC_FP64 if prec == "fp64" else hm.PREC_MIXED
    torch.cuda.synchronize()
    base = hm.device_bytes()
    failed = 0
    for k in (1, 2, 3, 5, 8, 13, 21, 34, 55, 89):
        hm.set_test_hook(hm.HOOK_FAIL_ALLOC, k)
        try:
            H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=p, symmetric=(prec == "mixed"))
        except hm.HMError as e:
            assert e.code == hm.ENOMEM, e
            assert "injected" in str(e)
            failed += 1
        else:
            H.free()                       # the build needed fewer allocations
        finally:
            hm.set_test_hook(hm.HOOK_FAIL_ALLOC, 0)
        torch.cuda.synchronize()
        assert hm.device_bytes() == base, k
    assert failed >= 5
    # the library still works
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=p)
    y = H.matvec(inputs.normal_vector(n, 1))
    H.free()
    assert np.isfinite(y).all()
    assert hm.device_bytes() == base


def _structure(hm, pts, cols=None, **kw):
    if cols is None:
        H = hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6, structure_only=True, **kw)
    else:
        H = hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6, structure_only=True, cols=cols, **kw)
    st, reruns = H.structure(), H.stats()["traversal_reruns"]
    H.free()
    return st, reruns


@pytest.mark.parametrize("case", ["uniform1d", "mixture2d", "uniform3d", "rect3d"])
def test_traversal_overflow_reruns_transparently(hm, case):
    d = {"uniform1d": 1, "mixture2d": 2, "uniform3d": 3, "rect3d": 3}[case]
    n = 1 << 14
    pts = (inputs.mixture_points(n, d, 31) if case == "mixture2d"
           else inputs.uniform_points(n, d, 31))
    cols = inputs.uniform_points(n // 2 + 77, d, 32) if case == "rect3d" else None
    ref, r0 = _structure(hm, pts, cols)
    assert r0 == 0                          # the default bounds fit
    hm.set_test_hook(hm.HOOK_TRAVERSAL_KAPPA, 1)
    try:
        got, r1 = _structure(hm, pts, cols)
    finally:
        hm.set_test_hook(hm.HOOK_TRAVERSAL_KAPPA, 0)
    assert r1 >= 2, r1                      # the forced bound overflowed
    for k in ("adm", "dense", "perm"):
        assert np.array_equal(got[k], ref[k]), k


def test_traversal_overflow_reports_eoverflow(hm):
    import torch
    pts = inputs.mixture_points(1 << 14, 2, 33)
    torch.cuda.synchronize()
    base = hm.device_bytes()
    hm.set_test_hook(hm.HOOK_TRAVERSAL_KAPPA, 1)
    hm.set_test_hook(hm.HOOK_TRAVERSAL_TRIES, 1)
    try:
        with pytest.raises(hm.HMError) as ei:
            hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6)
        assert ei.value.code == hm.EOVERFLOW
    finally:
        hm.set_test_hook(hm.HOOK_TRAVERSAL_TRIES, 0)
        hm.set_test_hook(hm.HOOK_TRAVERSAL_KAPPA, 0)
    torch.cuda.synchronize()
    assert hm.device_bytes() == base
    H = hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6)
    assert H.stats()["traversal_reruns"] == 0
    H.free()

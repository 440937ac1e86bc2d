"""The three calls of the boundary as a C caller makes them: hm_build,
hm_matvec and hm_free on plain host (numpy) buffers, no options struct, no
torch. The product must match the CPU oracle's H-matrix within 1e-10 (FP64,
the default arithmetic), with sigma^2 added on the diagonal; bad arguments
must come back as NULL / HM_EINVAL with a message, and hm_free(NULL) must be
harmless."""
import ctypes as C

import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm
    build.build()
    return hm.lib()


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


@pytest.mark.parametrize("n,d,kernel,ell,leaf,eta,eps,sigma2", [
    (4096, 2, 0, 0.1, 32, 1.0, 1e-8, 0.0),
    (3000, 3, 1, 0.2, 48, 1.0, 1e-8, 0.01),
    (1, 2, 0, 0.1, 32, 1.0, 1e-8, 0.5),
])
def test_bare_build_matvec_free(L, orc, n, d, kernel, ell, leaf, eta, eps, sigma2):
    pts = np.ascontiguousarray(inputs.uniform_points(n, d, 41))
    x = np.ascontiguousarray(inputs.normal_vector(n, inputs.X_SEED))
    y = np.zeros(n)
    prm = np.array([ell, sigma2])
    h = L.hm_build(_p(pts), n, d, kernel, _p(prm), leaf, eta, eps)
    assert h, L.hm_last_error()
    try:
        assert L.hm_matvec(h, _p(x), _p(y)) == 0, L.hm_last_error()
        # a second product into the same buffer overwrites it
        y2 = np.full(n, 7.0)
        assert L.hm_matvec(h, _p(x), _p(y2)) == 0
    finally:
        L.hm_free(h)
    O = orc.HMatrix(pts, kernel, ell, leaf, eta, eps, sigma2=sigma2)
    yo = O.matvec(x)
    err = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    assert err <= 1e-10, err
    assert np.array_equal(y, y2)


def test_bare_calls_reject_bad_arguments(L):
    pts = np.ascontiguousarray(inputs.uniform_points(100, 2, 3))
    prm = np.array([0.1, 0.0])
    assert not L.hm_build(_p(pts), 100, 4, 0, _p(prm), 32, 1.0, 1e-6)   # d = 4
    assert b"d" in L.hm_last_error()
    bad = np.array([-1.0, 0.0])
    assert not L.hm_build(_p(pts), 100, 2, 0, _p(bad), 32, 1.0, 1e-6)   # l <= 0
    assert not L.hm_build(_p(pts), 0, 2, 0, _p(prm), 32, 1.0, 1e-6)     # N = 0
    nanpts = pts.copy()
    nanpts[5, 1] = np.nan
    assert not L.hm_build(_p(nanpts), 100, 2, 0, _p(prm), 32, 1.0, 1e-6)
    y = np.zeros(100)
    assert L.hm_matvec(None, _p(y), _p(y)) == -1
    L.hm_free(None)

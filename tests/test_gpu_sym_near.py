"""Symmetric near field (hm_options.symmetric = 2).

Both kernels are symmetric, so a dense leaf (sigma, tau) is the transpose of
(tau, sigma). With symmetric = 2 a mixed-precision build stores only the
dense leaves with tau.lo <= sigma.lo; the product's gather applies every
off-diagonal one both ways (A x|sigma into the rows of tau, A^T x|tau into
the rows of sigma, the latter through a per-column buffer summed by the
finish in a fixed order). The near field's bytes about halve; the product
must stay within the mixed tolerance of the oracle's mirrored H-matrix, agree
with the symmetric = 1 product to rounding, and keep every determinism
property of the product (launch shapes, CUDA graphs, several right-hand
sides, block-row shares, batches)."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import dist, inputs

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def hm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm as H
    build.build()
    H.lib()
    yield H
    H.set_gather_shape(-1)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [
    # n, d, points, kernel, ell, leaf, eta, sigma2
    (1 << 15, 2, "m", 0, 0.1, 64, 1.0, 0.0),      # the benchmark's mixture
    (20000, 3, "u", 1, 0.2, 48, 1.0, 0.01),       # Matern-3/2, ragged tiles, shift
    (7000, 1, "u", 0, 0.05, 32, 1.5, 0.0),        # 1-D
    (50, 2, "u", 0, 0.3, 64, 1.0, 0.1),           # one leaf: only the diagonal block
]


def _pts(n, d, kind, seed=61):
    return inputs.uniform_points(n, d, seed) if kind == "u" else inputs.mixture_points(n, d, seed)


@pytest.mark.parametrize("case", CASES)
def test_symmetric_near_field_matches_oracle(hm, orc, case):
    n, d, kind, kern, ell, leaf, eta, s2 = case
    pts = _pts(n, d, kind)
    x = inputs.normal_vector(n, inputs.X_SEED)
    kw = dict(precision=hm.PREC_MIXED, sigma2=s2)
    H1 = hm.HMatrix(pts, kern, ell, leaf, eta, 1e-6, symmetric=1, **kw)
    H2 = hm.HMatrix(pts, kern, ell, leaf, eta, 1e-6, symmetric=2, **kw)
    y1, y2 = H1.matvec(x), H2.matvec(x)
    s1, s2s = H1.stats(), H2.stats()
    H1.free()
    H2.free()
    O = orc.HMatrix(pts, kern, ell, leaf, eta, 1e-6, sigma2=s2, symmetric=True)
    assert rel(y2, O.matvec(x)) <= MIXED_TOL
    assert rel(y2, y1) <= 1e-6
    # the same leaves and ranks; the near field about halves (in 1-D a leaf
    # has two off-diagonal dense partners, so the diagonal keeps a third)
    assert s2s["n_dense"] == s1["n_dense"] and s2s["sum_rank"] == s1["sum_rank"]
    if n > leaf:
        assert s2s["near_bytes"] <= (0.7 if d == 1 else 0.6) * s1["near_bytes"]
        assert s2s["mvp_bytes"] < s1["mvp_bytes"]
    else:
        assert s2s["near_bytes"] == s1["near_bytes"]


def test_launch_shapes_and_repeats_are_bit_identical(hm):
    n = 1 << 15
    pts = _pts(n, 2, "m", 62)
    x = inputs.normal_vector(n, 3)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED, symmetric=2)
    try:
        ref = H.matvec(x)
        for shape in (0, 1, 2, 3, 4, -1):
            hm.set_gather_shape(shape)
            assert np.array_equal(H.matvec(x), ref), shape
        hm.set_batch_limits(0, 5)
        assert np.array_equal(H.matvec(x), ref)
    finally:
        hm.set_gather_shape(-1)
        hm.set_batch_limits(0, 0)
    H.free()


def test_several_vectors_and_graph_replay(hm):
    import torch
    n = 1 << 14
    pts = torch.from_numpy(_pts(n, 2, "m", 63)).cuda()
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED, symmetric=2,
                   sigma2=0.01)
    X = inputs.normal_vector(n, 4, nrhs=5)
    Y = H.matvec(X)
    for r in range(5):
        assert np.array_equal(Y[r], H.matvec(X[r]))
    x = torch.from_numpy(X[0]).cuda()
    ref = H.matvec(x)
    torch.cuda.synchronize()
    xs = x.clone()
    ys = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        H.matvec(xs, ys, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ys, ref)
    H.free()


def test_row_shares_give_the_rows_bit_for_bit(hm):
    n = 1 << 15
    pts = _pts(n, 2, "m", 64)
    x = inputs.normal_vector(n, 5)
    kw = dict(precision=hm.PREC_MIXED, symmetric=2, sigma2=0.01)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, **kw)
    y = H.matvec(x)
    st = H.structure()
    lo, hi, _, _ = H.tree()
    H.free()
    for r0, r1 in dist.shard_rows(lo, hi, st["adm"], st["dense"], n, 3):
        Hp = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, row_range=(r0, r1), **kw)
        yp = Hp.matvec(x)
        Hp.free()
        rows = st["perm"][r0:r1]
        assert np.array_equal(yp[rows], y[rows]), (r0, r1)


def test_batch_equals_separate_builds(hm):
    sets = [_pts(9000, 2, "m", 65), _pts(5000, 3, "u", 66)]
    kw = dict(precision=hm.PREC_MIXED, symmetric=2)
    B = hm.HBatch(sets, 0, 0.1, 64, 1.0, 1e-6, **kw)
    xs = [inputs.normal_vector(p.shape[0], 7 + q) for q, p in enumerate(sets)]
    y = B.matvec(np.concatenate(xs))
    B.free()
    o = 0
    for p, xq in zip(sets, xs):
        H = hm.HMatrix(p, 0, 0.1, 64, 1.0, 1e-6, **kw)
        assert rel(y[o:o + len(xq)], H.matvec(xq)) <= 1e-12
        H.free()
        o += len(xq)


def test_fp64_and_other_formats_fall_back_to_symmetric_1(hm):
    n = 6000
    pts = _pts(n, 2, "m", 67)
    x = inputs.normal_vector(n, 8)
    for kw in (dict(precision=hm.PREC_FP64), dict(precision=hm.PREC_MIXED, near_format=hm.NEAR_BF16)):
        H1 = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, symmetric=1, **kw)
        H2 = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, symmetric=2, **kw)
        assert np.array_equal(H1.matvec(x), H2.matvec(x))
        assert H1.stats()["near_bytes"] == H2.stats()["near_bytes"]
        H1.free()
        H2.free()
    with pytest.raises(hm.HMError):
        hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, symmetric=3)

"""The product (Alg. 3, batched: Sec. 5.4) captured in a CUDA graph.

After its first call on a device (which times the gather's launch shapes and
keeps the fastest), the product on device buffers is a fixed sequence of
kernel launches on the caller's stream with no host synchronisation and no
allocation, so a caller can capture it once and replay it. A replay must give
bit for bit the uncaptured product, for a new x written into the captured
input buffer too; likewise the product with several right-hand sides and the
product of a batch of independent point sets (one graph for all sets)."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm
    build.build()
    hm.lib()
    return torch, hm


def _capture(torch, fn, stream):
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
        fn()
    return g


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_captured_product_replays_bit_for_bit(env, prec):
    torch, hm = env
    n = 1 << 15
    pts = torch.from_numpy(inputs.mixture_points(n, 2, 11)).cuda()
    p = hm.PREC_FP64 if prec == "fp64" else hm.PREC_MIXED
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=p, symmetric=(prec == "mixed"))
    x1 = torch.from_numpy(inputs.normal_vector(n, 1)).cuda()
    x2 = torch.from_numpy(inputs.normal_vector(n, 2)).cuda()
    ref1, ref2 = H.matvec(x1), H.matvec(x2)          # the first call also tunes
    torch.cuda.synchronize()
    xs = x1.clone()
    ys = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = _capture(torch, lambda: H.matvec(xs, ys, stream=s), s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ys, ref1)
    xs.copy_(x2)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ys, ref2)
    H.free()


def test_captured_multi_rhs_product(env):
    torch, hm = env
    n, nr = 1 << 14, 12
    pts = torch.from_numpy(inputs.uniform_points(n, 2, 12)).cuda()
    H = hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6, precision=hm.PREC_MIXED)
    X = torch.from_numpy(inputs.normal_vector(n, 3, nrhs=nr)).cuda()
    ref = H.matvec(X)
    torch.cuda.synchronize()
    Y = torch.zeros_like(X)
    s = torch.cuda.Stream()
    g = _capture(torch, lambda: H.matvec(X, Y, stream=s), s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(Y, ref)
    H.free()


def test_captured_batch_product(env):
    # a ragged batch of independent sets (sizes log-uniform, d in {2, 3}):
    # one graph replays the product of every set
    torch, hm = env
    rng = np.random.default_rng(5)
    sizes = np.round(np.exp(rng.uniform(np.log(2000), np.log(20000), 6))).astype(np.int64)
    dims = rng.integers(2, 4, 6).astype(np.int32)
    sets = [inputs.uniform_points(int(m), int(d), 100 + k) for k, (m, d) in enumerate(zip(sizes, dims))]
    s = torch.cuda.Stream()
    B = hm.HBatch(sets, 0, 0.15, 64, 1.0, 1e-6, precision=hm.PREC_MIXED, stream=s)
    x = torch.from_numpy(inputs.normal_vector(int(sizes.sum()), 4)).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        ref = B.matvec(x)
    torch.cuda.synchronize()
    y = torch.zeros_like(x)
    g = _capture(torch, lambda: B.matvec(x, y), s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    B.free()

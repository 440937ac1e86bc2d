"""GPU parity of the rank-model MLP kernels, CG and the batched build."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm as H
    build.build()
    H.lib()
    return H


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _theta(seed=3):
    from paper_1708_09707_gb300 import rank_model
    th = rank_model.init_theta(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    th[512:576] = 0.1 * rng.standard_normal(64)
    th[4672:4736] = 0.1 * rng.standard_normal(64)
    return th


def test_mlp_forward_and_gradient_match_oracle(hm, orc):
    import torch
    rng = np.random.default_rng(0)
    th = _theta()
    F = rng.standard_normal((3000, 8)).astype(np.float32).astype(np.float64)
    T = rng.standard_normal(3000)
    yo = orc.mlp_forward(th, F)
    lo, go = orc.mlp_loss_grad(th, F, T)
    thd = torch.from_numpy(th.astype(np.float32)).cuda()
    Fd = torch.from_numpy(F.astype(np.float32)).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    out = torch.empty(3000, dtype=torch.float32, device="cuda")
    hm.mlp_forward(thd, Fd, out)
    assert _rel(out.cpu().numpy().astype(np.float64), yo) <= 1e-5
    g = torch.empty(hm.MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    hm.mlp_loss_grad(thd, Fd, Td, g, loss)
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    assert _rel(g.cpu().numpy().astype(np.float64), go) <= 1e-4
    # every parameter block separately (W1, b1, W2, b2, W3, b3)
    gg = g.cpu().numpy().astype(np.float64)
    for a, b in ((0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 4800), (4800, 4801)):
        assert _rel(gg[a:b], go[a:b]) <= 1e-4, (a, b)


def test_adam_steps_match_oracle(hm, orc):
    import torch
    rng = np.random.default_rng(1)
    th = _theta(5)
    tho = th.copy()
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    thd = torch.from_numpy(th.astype(np.float32)).cuda()
    md = torch.zeros_like(thd)
    vd = torch.zeros_like(thd)
    for t in range(1, 6):
        grad = rng.standard_normal(th.size)
        orc.adam_step(tho, grad, m, v, t, lr=1e-3)
        hm.mlp_adam(thd, torch.from_numpy(grad.astype(np.float32)).cuda(), md, vd, t, lr=1e-3)
    assert np.allclose(thd.cpu().numpy(), tho, rtol=0, atol=1e-6)


def test_block_features_match_oracle(hm, orc):
    pts = inputs.uniform_points(5000, 3, 31)
    H = hm.HMatrix(pts, 1, 0.2, 32, 1.0, 1e-6)
    O = orc.HMatrix(pts, 1, 0.2, 32, 1.0, 1e-6)
    F, T = H.features()
    Fo = O.features()
    assert F.shape == Fo.shape
    assert np.allclose(F, Fo, rtol=1e-6, atol=1e-6)
    ro, _ = O.ranks()
    assert np.allclose(T, np.log2(1.0 + ro), rtol=0, atol=1e-6 + 0.0) or \
        np.mean(np.abs(T - np.log2(1.0 + ro)) > 1e-6) < 1e-3


def test_rank_model_trains_and_sizes_the_build(hm):
    """What the trained model gains: one compression pass without scratch
    copies, far less reserved factor memory, the same product."""
    from paper_1708_09707_gb300 import rank_model
    sets = (dict(points="mixture", n=1 << 16, d=2, kernel=0, ell=0.1, leaf=64, eta=1.0,
                 eps=1e-6, adm_max=False, seed=1203),
            dict(points="uniform", n=1 << 15, d=3, kernel=1, ell=0.2, leaf=64, eta=1.0,
                 eps=1e-6, adm_max=False, seed=1202))
    F, T = rank_model.training_data(sets)
    theta, hist = rank_model.train(F, T, epochs=12, batch=8192, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    pts = inputs.mixture_points(1 << 17, 2, 1303)      # unseen set, larger
    x = inputs.normal_vector(1 << 17, 9)
    plain = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED)
    learned = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED,
                         rank_model_theta=theta)
    sp, sl = plain.stats(), learned.stats()
    assert _rel(learned.matvec(x), plain.matvec(x)) <= 1e-5
    # all blocks converged: mispredicted ones were re-run with the full cap
    assert sl["rank_cap_hits"] == 0
    assert sl["n_mispredicted"] <= 0.10 * sl["n_adm"], sl["n_mispredicted"]
    assert sl["reserved_factor_entries"] < 0.5 * sp["reserved_factor_entries"]
    assert sl["aca_passes"] <= 2


@pytest.mark.parametrize("sigma2", [1e-1, 1e-2])
def test_cg_matches_oracle(hm, orc, sigma2):
    n = 3000
    pts = inputs.uniform_points(n, 2, 41)
    b = inputs.normal_vector(n, inputs.CG_SEED)
    H = hm.HMatrix(pts, 1, 0.1, 32, 1.0, 1e-8, sigma2=sigma2)
    O = orc.HMatrix(pts, 1, 0.1, 32, 1.0, 1e-8, sigma2=sigma2)
    x, it, rr = H.cg(b, rtol=1e-8, maxit=3000)
    xo, ito, rro = O.cg(b, rtol=1e-8, maxit=3000)
    # CG in finite precision: the two products differ in rounding order, so on
    # an ill-conditioned system the iteration counts drift apart by a few
    assert rr <= 1e-8 and abs(it - ito) <= max(2, 0.02 * ito), (it, ito)
    assert _rel(x, xo) <= 1e-6
    # the true residual with a fresh product
    assert _rel(H.matvec(x), b) <= 2e-8
    # mixed precision operator: it converges on its own residual; its solution
    # has a small normwise backward error in the FP64 system,
    # |b - A xm| / (|A| |xm| + |b|), since the operator's entries are accurate
    # to about 1e-5 of |A|; the forward error is at most the condition number
    # (|A| / sigma^2, the kernel matrix being positive semidefinite) times it
    Hm = hm.HMatrix(pts, 1, 0.1, 32, 1.0, 1e-8, sigma2=sigma2, precision=hm.PREC_MIXED)
    xm, itm, rrm = Hm.cg(b, rtol=1e-6, maxit=3000)
    assert rrm <= 1e-6
    v = b / np.linalg.norm(b)
    for _ in range(30):                                   # power iteration, |A|_2
        w = H.matvec(v)
        nrm = float(np.linalg.norm(w))
        v = w / nrm
    back = np.linalg.norm(b - H.matvec(xm)) / (nrm * np.linalg.norm(xm) + np.linalg.norm(b))
    assert back <= 1e-5, back
    assert _rel(xm, xo) <= 4.0 * back * nrm / sigma2
    # the same with the symmetric product (symmetric = 2), the benchmark's form
    Hs = hm.HMatrix(pts, 1, 0.1, 32, 1.0, 1e-8, sigma2=sigma2, precision=hm.PREC_MIXED,
                    symmetric=2)
    xs, its, rrs = Hs.cg(b, rtol=1e-6, maxit=3000)
    assert rrs <= 1e-6
    backs = np.linalg.norm(b - H.matvec(xs)) / (nrm * np.linalg.norm(xs) + np.linalg.norm(b))
    assert backs <= 1e-5, backs
    Hs.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_separate_builds(hm, prec):
    sizes, dims = inputs.ragged_batch_sizes(6, 77, lo=2000, hi=20000)
    sets = [inputs.uniform_points(int(s), int(d), 500 + q) for q, (s, d) in enumerate(zip(sizes, dims))]
    B = hm.HBatch(sets, 0, 0.15, 64, 1.0, 1e-6, precision=prec)
    xs = [inputs.normal_vector(p.shape[0], 600 + q) for q, p in enumerate(sets)]
    y = B.matvec(np.concatenate(xs))
    o = 0
    for q, p in enumerate(sets):
        H = hm.HMatrix(p, 0, 0.15, 64, 1.0, 1e-6, precision=prec)
        yq = H.matvec(xs[q])
        assert np.array_equal(y[o:o + p.shape[0]], yq), q
        o += p.shape[0]
    st = B.stats()
    assert st["n_points"] == int(sizes.sum())


def test_alu_peak_is_plausible(hm):
    """The measured FMA peaks used as roofline denominators: FP32 near the
    CUDA-core rate, FP64 far below it on this part."""
    f32 = hm.alu_peak(hm.PREC_MIXED)
    f64 = hm.alu_peak(hm.PREC_FP64)
    assert 10e12 < f32 < 200e12, f32
    assert 0.1e12 < f64 < f32, f64
    with pytest.raises(hm.HMError):
        hm.alu_peak(7)

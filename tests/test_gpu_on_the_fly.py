"""The on-the-fly product (no stored factors or near field; ACA and the dense
leaves recomputed inside every product): equal to the oracle within the
FP64 / mixed bounds, equal to the stored product to rounding, and the same
bits whatever the number of ACA passes."""
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
    return H


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _pts(n, d, kind, seed):
    if kind == "m":
        return inputs.mixture_points(n, d, seed)
    return inputs.uniform_points(n, d, seed)


@pytest.mark.parametrize("case", [(6000, 2, "m", 0, 0.1, 64, 1.0, 1e-8, False),
                                  (5000, 3, "u", 1, 0.2, 32, 1.0, 1e-6, False),
                                  (4096, 2, "u", 0, 0.1, 32, 1.0, 1e-8, True)],
                         ids=["mix2d", "matern3d", "uniform2d_max"])
def test_fp64_matches_oracle_and_stored(hm, orc, case):
    n, d, kind, kern, ell, leaf, eta, eps, adm_max = case
    pts = _pts(n, d, kind, 11)
    x = inputs.normal_vector(n, inputs.X_SEED)
    H = hm.HMatrix(pts, kern, ell, leaf, eta, eps, sigma2=0.01, adm_max=adm_max, on_the_fly=True)
    y = H.matvec(x)
    O = orc.HMatrix(pts, kern, ell, leaf, eta, eps, sigma2=0.01, adm_max=adm_max)
    assert rel(y, O.matvec(x)) <= FP64_TOL
    S = hm.HMatrix(pts, kern, ell, leaf, eta, eps, sigma2=0.01, adm_max=adm_max)
    # the same ACA factors; only the order of the row sums differs
    assert rel(y, S.matvec(x)) <= 1e-13
    assert np.array_equal(H.matvec(x), y)
    st = H.stats()
    # nothing stored; the dense entries are evaluated in every product
    assert st["factor_entries"] == 0 and st["factor_bytes"] == 0 and st["near_bytes"] == 0
    assert st["near_entries"] == S.stats()["near_entries"]
    assert np.array_equal(H.structure()["adm"], S.structure()["adm"])


@pytest.mark.parametrize("prec", [0, 1])
def test_pass_count_does_not_change_bits(hm, prec):
    n = 20000
    pts = _pts(n, 2, "m", 21)
    x = inputs.normal_vector(n, 3)
    H1 = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=prec, on_the_fly=True)
    H2 = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=prec, on_the_fly=True,
                    scratch_gb=0.004)
    assert H1.stats()["aca_passes"] == 1
    assert H2.stats()["aca_passes"] > 2
    assert np.array_equal(H1.matvec(x), H2.matvec(x))


def test_mixed_matches_oracle_and_options(hm, orc):
    import torch
    n = 9000
    pts = _pts(n, 2, "m", 31)
    x = inputs.normal_vector(n, 5)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, sigma2=0.25, precision=hm.PREC_MIXED,
                   on_the_fly=True)
    y = H.matvec(x)
    O = orc.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, sigma2=0.25)
    assert rel(y, O.matvec(x)) <= MIXED_TOL
    yd = H.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y, yd)
    X = np.stack([x, -2 * x, inputs.normal_vector(n, 6)])
    Y = H.matvec(X)
    for r in range(3):
        assert np.array_equal(Y[r], H.matvec(X[r]))
    Ha = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, sigma2=0.25, precision=hm.PREC_MIXED,
                    on_the_fly=True, accumulate=True)
    ya = np.ones(n)
    Ha.matvec(x, ya)
    assert np.array_equal(ya, y + 1.0)


@pytest.mark.parametrize("sym", [False, True], ids=["general", "symmetric"])
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_on_the_fly(hm, orc, prec, sym):
    """hm_build_batch with on_the_fly: the passes run over the leaves of all
    sets in order, so one pass may hold leaves of several sets. Every set's
    part of the product equals the oracle's H-matrix of that set within the
    FP64 / mixed bound and that set's own on-the-fly product to rounding, the
    stored batch's product agrees, and a repeated product gives the same
    bits."""
    # uniform sets: on a 4000-point mixture the FP32 kernel entries alone put
    # the mixed product 1.4e-5 from the FP64 one (every mixed storage mode alike)
    sets = [_pts(4000, 2, "u", 42), _pts(3000, 3, "u", 43), _pts(2500, 1, "u", 44),
            _pts(40, 3, "u", 45)]
    eps = 1e-8 if prec == 0 else 1e-6
    kw = dict(precision=prec, symmetric=sym, sigma2=0.01)
    xs = [inputs.normal_vector(p.shape[0], 50 + q) for q, p in enumerate(sets)]
    x = np.concatenate(xs)
    B = hm.HBatch(sets, 0, 0.1, 32, 1.0, eps, on_the_fly=True, scratch_gb=0.004, **kw)
    y = B.matvec(x)
    st = B.stats()
    assert st["aca_passes"] > 2
    assert st["factor_bytes"] == 0 and st["near_bytes"] == 0
    assert np.array_equal(B.matvec(x), y)
    B.free()
    S = hm.HBatch(sets, 0, 0.1, 32, 1.0, eps, **kw)
    ys = S.matvec(x)
    S.free()
    assert rel(y, ys) <= (1e-13 if prec == 0 else MIXED_TOL)
    o = 0
    for p, xq in zip(sets, xs):
        yq = y[o:o + len(xq)]
        O = orc.HMatrix(p, 0, 0.1, 32, 1.0, eps, sigma2=0.01, symmetric=sym)
        assert rel(yq, O.matvec(xq)) <= (FP64_TOL if prec == 0 else MIXED_TOL)
        H = hm.HMatrix(p, 0, 0.1, 32, 1.0, eps, on_the_fly=True, **kw)
        assert rel(yq, H.matvec(xq)) <= 1e-13
        H.free()
        o += len(xq)


def test_refused_combinations(hm):
    pts = _pts(500, 2, "u", 41)
    with pytest.raises(hm.HMError):
        hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6, cols=pts, precision=hm.PREC_MIXED,
                   on_the_fly=True, rank_model_theta=np.zeros(4801, np.float32))


@pytest.fixture(scope="module")
def theta(hm):
    from paper_1708_09707_gb300 import rank_model
    F, T = rank_model.training_data()
    th, _ = rank_model.train(F, T)
    return th


@pytest.mark.parametrize("sym", [False, True])
def test_rank_model_on_the_fly(hm, orc, theta, sym):
    # the learned model sizes each pass's reservations; blocks predicted too
    # small run again inside their pass: the product is that of the stored
    # build with the model, to the mixed bound against the oracle
    n = 1 << 15
    w = inputs.WORKLOADS["matern3d_n1m"]
    pts = inputs.workload_points("matern3d_n1m", n)
    x = inputs.normal_vector(n, inputs.X_SEED)
    O = orc.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], symmetric=sym)
    yo = O.matvec(x)
    kw = dict(precision=hm.PREC_MIXED, symmetric=sym, rank_model_theta=theta)
    Hp = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], on_the_fly=True,
                    scratch_gb=0.05, **kw)
    Hf = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], on_the_fly=True,
                    scratch_gb=0.05, symmetric=sym, precision=hm.PREC_MIXED)
    assert Hp.stats()["aca_passes"] < Hf.stats()["aca_passes"]
    y = Hp.matvec(x)
    st = Hp.stats()
    assert rel(y, yo) <= MIXED_TOL, rel(y, yo)
    assert st["n_mispredicted"] <= 0.05 * st["n_adm"]
    Hs = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                    near_format=hm.NEAR_FP32, **kw)
    assert rel(y, Hs.matvec(x)) <= 1e-6
    for H in (Hp, Hf, Hs):
        H.free()


def test_rank_model_on_the_fly_forced_reruns(hm, orc):
    # a model that predicts rank 1 for every block: nearly every block runs
    # twice, and the product still meets the FP64 bound
    n = 6000
    pts = _pts(n, 2, "m", 43)
    x = inputs.normal_vector(n, inputs.X_SEED)
    th = np.zeros(4801, np.float32)
    th[4800] = -4.0                      # yhat = -4: the smallest reservation
    O = orc.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-8)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-8, on_the_fly=True, rank_model_theta=th)
    y = H.matvec(x)
    st = H.stats()
    H.free()
    assert rel(y, O.matvec(x)) <= FP64_TOL
    assert st["n_mispredicted"] > 0.5 * st["n_adm"]


def test_rank_model_tight_scratch_with_large_blocks(hm, orc):
    # every pass filled to a small scratch, blocks above 2048 rows (whose
    # reservation has a floor of 32 ranks) predicted at rank 1: the passes
    # are cut by the reservations the ACA then uses, so each fits its scratch
    n = 6000
    pts = _pts(n, 2, "m", 44)
    x = inputs.normal_vector(n, inputs.X_SEED)
    th = np.zeros(4801, np.float32)
    th[4800] = -4.0
    O = orc.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-8)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-8, on_the_fly=True, rank_model_theta=th,
                   scratch_gb=0.002)
    y = H.matvec(x)
    st = H.stats()
    H.free()
    assert st["aca_passes"] >= 3
    assert rel(y, O.matvec(x)) <= FP64_TOL


def test_no_admissible_leaf_and_eta_zero(hm, orc):
    """C >= N leaves one dense block and eta = 0 admits no block of positive
    diameter: both products are the dense matrix-vector product."""
    pts = _pts(300, 2, "u", 51)
    x = inputs.normal_vector(300, 8)
    truth = orc.dense_matvec(pts, 0, 0.1, 0.0, x)
    H = hm.HMatrix(pts, 0, 0.1, 512, 1.0, 1e-8, on_the_fly=True)
    assert H.stats()["n_adm"] == 0
    assert rel(H.matvec(x), truth) <= 1e-13
    pts = _pts(2000, 2, "u", 52)
    x = inputs.normal_vector(2000, 9)
    H = hm.HMatrix(pts, 0, 0.1, 16, 0.0, 1e-8, on_the_fly=True)
    assert rel(H.matvec(x), orc.dense_matvec(pts, 0, 0.1, 0.0, x)) <= 1e-13


def test_cg_with_on_the_fly_products(hm, orc):
    """CG on (A + sigma^2 I) with an on-the-fly handle: every iteration
    recomputes the H-matrix; the solution matches the oracle's CG."""
    n = 3000
    pts = inputs.uniform_points(n, 2, 41)
    b = inputs.normal_vector(n, inputs.CG_SEED)
    H = hm.HMatrix(pts, 1, 0.1, 32, 1.0, 1e-8, sigma2=0.1, on_the_fly=True)
    O = orc.HMatrix(pts, 1, 0.1, 32, 1.0, 1e-8, sigma2=0.1)
    x, it, rr = H.cg(b, rtol=1e-8, maxit=3000)
    xo, ito, rro = O.cg(b, rtol=1e-8, maxit=3000)
    assert rr <= 1e-8 and abs(it - ito) <= max(2, 0.02 * ito), (it, ito)
    assert rel(x, xo) <= 1e-6
    assert rel(H.matvec(x), b) <= 2e-8
    with pytest.raises(hm.HMError):
        H.factors(0, 32, 32)


def test_profiled_phases(hm):
    """profile = 1 on an on-the-fly handle: per-phase CUDA-event times summed
    over the products since the last hm_get_stats, the ACA work of one product
    counted, and the product unchanged by the profiling."""
    pts = _pts(8000, 2, "m", 21)
    x = inputs.normal_vector(8000, 22)
    P = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED, on_the_fly=True,
                   profile=True, scratch_gb=0.01)
    Q = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, precision=hm.PREC_MIXED, on_the_fly=True,
                   scratch_gb=0.01)
    y = P.matvec(x)
    P.matvec(x)
    assert np.array_equal(y, Q.matvec(x))
    st = P.stats()
    assert st["mvp_count"] == 2 and st["aca_passes"] > 1
    parts = st["t_np_aca_ms"] + st["t_np_lowrank_ms"] + st["t_np_near_ms"]
    assert min(st["t_np_aca_ms"], st["t_np_lowrank_ms"], st["t_np_near_ms"]) > 0
    # disjoint intervals inside the product (event times have about 0.5 us resolution)
    assert parts <= st["t_mvp_ms"] * 1.01 + 0.1
    assert st["aca_evals"] > 0 and st["aca_flops"] > 0 and st["sum_rank"] > 0
    assert st["near_entries"] > 0
    # the sums restart after hm_get_stats
    assert P.stats()["mvp_count"] == 0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", [(6000, 2, "m", 0, 0.1, 64, 1.0), (5000, 3, "u", 1, 0.2, 32, 1.0)],
                         ids=["mix2d", "matern3d"])
def test_symmetric_on_the_fly(hm, orc, case, prec):
    """Symmetric mode on the fly: each pass compresses the canonical leaves
    (tau.lo <= sigma.lo) of its block range and applies them and their mirror
    leaves (U and V exchanged); the product equals the stored symmetric one
    and the oracle's mirrored H-matrix, with about half the ACA work of the
    non-symmetric product."""
    n, d, kind, kern, ell, leaf, eta = case
    eps = 1e-8 if prec == 0 else 1e-6
    pts = _pts(n, d, kind, 11)
    x = inputs.normal_vector(n, inputs.X_SEED)
    kw = dict(precision=prec, symmetric=True)
    F = hm.HMatrix(pts, kern, ell, leaf, eta, eps, on_the_fly=True, profile=True,
                   scratch_gb=0.004, **kw)
    y = F.matvec(x)
    sf = F.stats()
    assert sf["aca_passes"] > 1
    O = orc.HMatrix(pts, kern, ell, leaf, eta, eps, symmetric=True)
    yo = O.matvec(x)
    if prec == 0:
        S = hm.HMatrix(pts, kern, ell, leaf, eta, eps, **kw)
        assert rel(y, S.matvec(x)) <= 1e-13
        assert rel(y, yo) <= FP64_TOL
        # a different pass count changes the order of the row sums only
        G = hm.HMatrix(pts, kern, ell, leaf, eta, eps, on_the_fly=True, scratch_gb=0.02, **kw)
        assert rel(G.matvec(x), y) <= 1e-14
    else:
        assert rel(y, yo) <= MIXED_TOL
    assert np.array_equal(F.matvec(x), y)
    N = hm.HMatrix(pts, kern, ell, leaf, eta, eps, on_the_fly=True, profile=True,
                   scratch_gb=0.004, precision=prec)
    N.matvec(x)
    sn = N.stats()
    assert sf["aca_evals"] < 0.65 * sn["aca_evals"], (sf["aca_evals"], sn["aca_evals"])

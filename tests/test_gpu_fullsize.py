"""GPU path at the benchmark sizes: integer structure bit-exact against the
oracle at N = 2^20, the largest blocks (thread-block-cluster ACA path)
against the oracle's ACA of the same blocks, and sampled rows of the product
against the brute-force sum."""
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


def _block_dims(lo, hi, leaves):
    return hi[leaves[:, 0]] - lo[leaves[:, 0]], hi[leaves[:, 1]] - lo[leaves[:, 1]]


def test_largest_blocks_match_oracle(hm, orc):
    # on a line, quarter-length clusters two apart are admissible: blocks of
    # 65536 and 32768 points run on clusters of 8 and 4 CTAs
    n = 1 << 18
    pts = inputs.uniform_points(n, 1, 21)
    H = hm.HMatrix(pts, 0, 0.05, 64, 1.5, 1e-8)
    O = orc.HMatrix(pts, 0, 0.05, 64, 1.5, 1e-8, compress=False)
    s = H.structure()
    A = O.adm_leaves()
    assert np.array_equal(s["adm"], A)
    lo, hi, _, _ = O.tree()
    m, nn = _block_dims(lo, hi, A)
    big = np.nonzero(np.maximum(m, nn) > 4096)[0]
    assert (np.maximum(m, nn)[big] > 32768).any() and (np.maximum(m, nn)[big] <= 32768).any()
    pick = list(big[np.argsort(-np.maximum(m, nn)[big])][:3]) + list(big[-2:])
    for b in pick:
        O.compress_range(int(b), int(b) + 1)
        Uo, Vo = O.factors(int(b))
        U, V = H.factors(int(b), int(m[b]), int(nn[b]))
        assert U.shape[1] == Uo.shape[1], (b, U.shape, Uo.shape)
        # compare U V^T through random probes (the blocks are too large to form)
        z = np.random.default_rng(int(b)).standard_normal(int(nn[b]))
        ref = Uo @ (Vo.T @ z)
        assert np.linalg.norm(U @ (V.T @ z) - ref) <= 1e-10 * np.linalg.norm(ref), b


@pytest.mark.parametrize("name", ["mix2d_n1m", "matern3d_n1m"])
def test_fullsize_structure_bit_exact(hm, orc, name):
    w = inputs.WORKLOADS[name]
    pts = inputs.workload_points(name)
    O = orc.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], compress=False)
    # the integer structure does not depend on the compression that follows
    Hm = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                    structure_only=True)
    with pytest.raises(hm.HMError):
        Hm.matvec(np.zeros(w["n"]))
    s = Hm.structure()
    assert np.array_equal(s["codes"], O.codes())
    assert np.array_equal(s["perm"], O.perm())
    assert np.array_equal(s["adm"], O.adm_leaves())
    assert np.array_equal(s["dense"], O.dense_leaves())
    lo, hi, bmin, bmax = Hm.tree()
    olo, ohi, obmin, obmax = O.tree()
    assert np.array_equal(lo, olo) and np.array_equal(bmin, obmin) and np.array_equal(bmax, obmax)
    # leaves tile I x I exactly once
    am, an = _block_dims(olo, ohi, s["adm"])
    dm, dn = _block_dims(olo, ohi, s["dense"])
    assert int((am * an).sum() + (dm * dn).sum()) == w["n"] ** 2


def test_fullsize_sampled_rows(hm, orc):
    name = "mix2d_n1m"
    w = inputs.WORKLOADS[name]
    pts = inputs.workload_points(name)
    x = inputs.normal_vector(w["n"], inputs.X_SEED)
    rows = np.sort(np.random.default_rng(0).choice(w["n"], 64, replace=False))
    yb = orc.dense_rows(pts, w["kernel"], w["ell"], 0.0, rows, x)
    for prec in (hm.PREC_FP64, hm.PREC_MIXED):
        H = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"], precision=prec)
        y = H.matvec(x)
        e = np.linalg.norm(y[rows] - yb) / np.linalg.norm(yb)
        assert e <= 10 * w["eps"], (prec, e)
        H.free()


def test_timed_configuration_parity(hm, orc):
    # exactly the configuration bench.py times: the clipped mixture at
    # N = 2^20, mixed precision, symmetric mode with the symmetric near field
    # (symmetric = 2), the learned rank model
    # trained as the bench trains it; 256 sampled rows against the exact sums
    # (Neumaier-compensated FP64 brute force), and the whole product against
    # the FP64 GPU build, whose parity with the oracle the smaller cases pin
    from paper_1708_09707_gb300 import rank_model
    name = "mix2d_n1m"
    w = inputs.WORKLOADS[name]
    pts = inputs.workload_points(name)
    x = inputs.normal_vector(w["n"], inputs.X_SEED)
    F, T = rank_model.training_data()
    theta, _ = rank_model.train(F, T)
    H = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                   precision=hm.PREC_MIXED, symmetric=2, rank_model_theta=theta)
    y = H.matvec(x)
    st = H.stats()
    H.free()
    # the symmetric near field really is on: the stored near field about halves
    H1 = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                    precision=hm.PREC_MIXED, symmetric=1, rank_model_theta=theta)
    y1 = H1.matvec(x)
    assert st["near_bytes"] <= 0.6 * H1.stats()["near_bytes"]
    H1.free()
    assert np.linalg.norm(y - y1) / np.linalg.norm(y1) <= 1e-6
    assert st["n_mispredicted"] < 0.01 * st["n_adm"]
    rows = np.sort(np.random.default_rng(1).choice(w["n"], 256, replace=False))
    yb = orc.dense_rows(pts, w["kernel"], w["ell"], 0.0, rows, x)
    e_rows = np.linalg.norm(y[rows] - yb) / np.linalg.norm(yb)
    assert e_rows <= 1e-5, e_rows
    H64 = hm.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                     precision=hm.PREC_FP64)
    y64 = H64.matvec(x)
    H64.free()
    e64 = np.linalg.norm(y - y64) / np.linalg.norm(y64)
    assert e64 <= 1e-5, e64
    # the FP64 build itself against the exact rows, at the accuracy eps asks
    e64_rows = np.linalg.norm(y64[rows] - yb) / np.linalg.norm(yb)
    assert e64_rows <= 10 * w["eps"], e64_rows

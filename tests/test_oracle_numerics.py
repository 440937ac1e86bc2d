"""Pins of the oracle's floating-point steps: ACA (Alg. 2), H-MVP (Alg. 3),
brute force, CG and the rank-model MLP."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs


def _lowrank(m, n, r, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((r, n))


@pytest.mark.parametrize("m,n,r", [(40, 30, 1), (64, 64, 5), (100, 37, 12),
                                   (20, 90, 20)])
def test_aca_recovers_exact_rank(orc, m, n, r):
    A = _lowrank(m, n, r, m + n + r)
    U, V, pi, pj, rej = orc.aca_dense(A, 1e-12, k_cap=64)
    assert U.shape[1] == r
    assert np.linalg.norm(A - U @ V.T) <= 1e-13 * np.linalg.norm(A) * max(1, r)
    # u_r is normalised so that its pivot entry is exactly one
    assert np.all(U[pi, np.arange(r)] == 1.0)
    # pivots are distinct
    assert len(set(pi)) == r and len(set(pj)) == r


def test_aca_cross_interpolation(orc):
    # the residual A - U V^T vanishes on the pivot rows and columns
    pts = inputs.uniform_points(300, 2, 3)
    X, Y = pts[:120], pts[150:] + np.array([1.5, 0.0])
    A = np.exp(-((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1) / 0.5 ** 2)
    U, V, pi, pj, _ = orc.aca_dense(A, 0.0, k_cap=6)   # fixed-rank mode
    assert U.shape[1] == 6
    R = A - U @ V.T
    scale = np.abs(A).max()
    assert np.abs(R[pi, :]).max() <= 1e-13 * scale
    assert np.abs(R[:, pj]).max() <= 1e-13 * scale


def test_aca_first_column_and_pivot_rule(orc):
    A = np.array([[1.0, 2.0, 3.0], [4.0, -8.0, 6.0], [2.0, 1.0, 0.5]])
    U, V, pi, pj, _ = orc.aca_dense(A, 0.0, k_cap=1)
    # first column j=0: |column| max at row 1 (value 4); u = col/4; v = row 1
    assert pj[0] == 0 and pi[0] == 1
    assert np.allclose(U[:, 0], [0.25, 1.0, 0.5])
    assert np.allclose(V[:, 0], [4.0, -8.0, 6.0])
    U, V, pi, pj, _ = orc.aca_dense(A, 0.0, k_cap=2)
    # second column: argmax over unused columns {1,2} of the reference row's
    # residual: row 0 minus u_1[0] v_1 = [1,2,3] - 0.25 [4,-8,6] = [0, 4, 1.5]
    assert pj[1] == 1
    B = np.array([[1.0, 2.0, 9.0], [4.0, -8.0, 6.0], [2.0, 1.0, 0.5]])
    U, V, pi, pj, _ = orc.aca_dense(B, 0.0, k_cap=2)
    # [1,2,9] - 0.25 [4,-8,6] = [0, 4, 7.5] -> column 2, although |v_1| is
    # largest at column 1
    assert pi[0] == 1 and pj[1] == 2


def test_aca_near_duplicate_columns(orc):
    # points on a line with a tight pair next to the first column: the
    # reference-row choice keeps the cross approximation accurate
    rng = np.random.default_rng(5)
    X = np.sort(rng.uniform(0, 1, 300))
    Y = np.concatenate([[2.0, 2.0 + 1e-9, 2.0 + 2e-9], rng.uniform(2.0, 4.0, 200)])
    A = np.exp(-(X[:, None] - Y[None, :]) ** 2 / 0.5)
    U, V, *_ = orc.aca_dense(A, 1e-8, k_cap=64)
    assert np.linalg.norm(A - U @ V.T) <= 10 * 1e-8 * np.linalg.norm(A)


def test_aca_rejects_zero_columns(orc):
    A = np.zeros((10, 6))
    A[:, 3] = np.arange(1, 11)
    A[:, 5] = 2 * np.arange(1, 11)
    U, V, pi, pj, rej = orc.aca_dense(A, 1e-10, k_cap=6)
    assert U.shape[1] == 1 and pj[0] == 3
    assert np.linalg.norm(A - U @ V.T) <= 1e-14 * np.linalg.norm(A)
    assert rej >= 3
    # an all-zero block has rank 0
    U, V, *_ = orc.aca_dense(np.zeros((5, 5)), 1e-6)
    assert U.shape[1] == 0


def test_aca_error_vs_svd_tail(orc):
    # Eckart-Young: ||A - UV^T||_F >= sqrt(sum_{i>r} s_i^2), and the adaptive
    # rule reaches eps relative accuracy on kernel blocks
    pts = inputs.uniform_points(400, 3, 5)
    X, Y = pts[:200], pts[200:] + np.array([2.0, 0.0, 0.0])
    for kern, ell in ((0, 1.0), (1, 0.5)):
        A = np.array([[orc.kernel_eval(kern, ell, x, y) for y in Y] for x in X])
        s = np.linalg.svd(A, compute_uv=False)
        tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1]) / np.linalg.norm(A)
        for eps in (1e-4, 1e-6, 1e-8):
            U, V, *_ = orc.aca_dense(A, eps, k_cap=128)
            r = U.shape[1]
            err = np.linalg.norm(A - U @ V.T)
            assert err >= np.sqrt((s[r:] ** 2).sum()) * (1 - 1e-9)
            assert r < 128
            assert err <= 10 * eps * np.linalg.norm(A), (kern, eps, r)
            # near-optimal rank: within 2x of the SVD rank at the same accuracy
            assert r <= 2 * int(np.argmax(tail < eps)), (kern, eps, r)


def test_kernel_closed_forms(orc):
    a = np.array([0.1, 0.2, 0.3])
    b = np.array([0.4, -0.2, 0.3])
    r2 = 0.09 + 0.16
    assert orc.kernel_eval(0, 0.5, a, b) == pytest.approx(np.exp(-r2 / 0.25), rel=1e-15)
    s = np.sqrt(3 * r2) / 0.5
    assert orc.kernel_eval(1, 0.5, a, b) == pytest.approx((1 + s) * np.exp(-s), rel=1e-15)
    assert orc.kernel_eval(1, 0.5, a, a) == 1.0
    assert orc.kernel_eval(0, 0.5, a, a) == 1.0


def test_dense_matvec_matches_numpy(orc):
    pts = inputs.uniform_points(300, 2, 9)
    x = inputs.normal_vector(300, 1)
    for kern in (0, 1):
        D2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
        if kern == 0:
            A = np.exp(-D2 / 0.1 ** 2)
        else:
            s = np.sqrt(3 * D2) / 0.1
            A = (1 + s) * np.exp(-s)
        y = orc.dense_matvec(pts, kern, 0.1, 0.3, x)
        assert np.allclose(y, A @ x + 0.3 * x, rtol=1e-13, atol=1e-13)
        rows = np.array([0, 17, 299])
        assert np.allclose(orc.dense_rows(pts, kern, 0.1, 0.3, rows, x), y[rows],
                           rtol=1e-15, atol=1e-15)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("d,kern", [(2, 0), (3, 1)])
def test_matvec_eta0_is_exact(orc, d, kern):
    pts = inputs.uniform_points(700, d, 21)
    x = inputs.normal_vector(700, 2)
    h = orc.HMatrix(pts, kern, 0.2, 16, 0.0, 1e-6)
    assert h.n_adm == 0
    assert _rel(h.matvec(x), orc.dense_matvec(pts, kern, 0.2, 0.0, x)) <= 1e-13


def test_matvec_single_dense_block(orc):
    pts = inputs.uniform_points(200, 2, 4)
    x = inputs.normal_vector(200, 3)
    h = orc.HMatrix(pts, 0, 0.3, 200, 1.0, 1e-6)
    assert h.n_adm == 0 and h.n_dense == 1
    assert _rel(h.matvec(x), orc.dense_matvec(pts, 0, 0.3, 0.0, x)) <= 1e-14


def test_matvec_config1_against_brute_force(orc):
    w = inputs.WORKLOADS["gauss2d_n4096"]
    pts = inputs.workload_points("gauss2d_n4096")
    x = inputs.normal_vector(w["n"], inputs.X_SEED)
    h = orc.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                    adm_max=True)
    y = h.matvec(x)
    yb = orc.dense_matvec(pts, w["kernel"], w["ell"], 0.0, x)
    e = _rel(y, yb)
    assert e <= 10 * w["eps"], e
    # sigma^2 shifts the result by sigma^2 x
    h2 = orc.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                     sigma2=0.5, adm_max=True)
    assert np.allclose(h2.matvec(x) - y, 0.5 * x, rtol=0, atol=1e-12)
    # symmetry of the operator up to the approximation error
    z = inputs.normal_vector(w["n"], 77)
    assert abs(z @ y - x @ h.matvec(z)) <= 10 * w["eps"] * np.linalg.norm(yb) * np.linalg.norm(z)


def test_symmetric_mirror_is_exactly_symmetric(orc):
    """Mirroring the transposed leaves (phi symmetric) makes the H-matrix
    symmetric to rounding, keeps it within the ACA accuracy of the dense
    product, and gives each mirror leaf the transposed factors of its
    partner (U and V exchanged, the same rank)."""
    w = inputs.WORKLOADS["gauss2d_n4096"]
    pts = inputs.workload_points("gauss2d_n4096")
    x = inputs.normal_vector(w["n"], inputs.X_SEED)
    z = inputs.normal_vector(w["n"], 77)
    h = orc.HMatrix(pts, w["kernel"], w["ell"], w["leaf"], w["eta"], w["eps"],
                    adm_max=True, symmetric=True)
    y = h.matvec(x)
    yb = orc.dense_matvec(pts, w["kernel"], w["ell"], 0.0, x)
    assert _rel(y, yb) <= 10 * w["eps"]
    hz = h.matvec(z)
    assert abs(z @ y - x @ hz) <= 1e-13 * np.linalg.norm(y) * np.linalg.norm(z)
    lo, hi, _, _ = h.tree()
    A = h.adm_leaves()
    r, _ = h.ranks()
    key = {(int(lo[t]), int(lo[s])): b for b, (t, s) in enumerate(A)}
    checked = 0
    for b, (t, s) in enumerate(A):
        if lo[t] <= lo[s] or checked >= 25:
            continue
        mb = key[(int(lo[s]), int(lo[t]))]
        U, V = h.factors(b)
        Um, Vm = h.factors(mb)
        assert r[b] == r[mb]
        assert np.array_equal(U, Vm) and np.array_equal(V, Um)
        checked += 1
    assert checked > 0


def test_matvec_fixed_rank_converges_geometrically(orc):
    # Sec. 6.4: e_rel decays exponentially in the fixed ACA rank k
    pts = inputs.uniform_points(2048, 2, 33)
    x = inputs.normal_vector(2048, 5)
    yb = orc.dense_matvec(pts, 0, 0.3, 0.0, x)
    errs = []
    for k in (1, 2, 4, 8, 12):
        h = orc.HMatrix(pts, 0, 0.3, 32, 1.5, 0.0, k_cap=k)
        errs.append(_rel(h.matvec(x), yb))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3 * errs[1], errs


def test_cg_matches_dense_solve(orc):
    n = 400
    pts = inputs.uniform_points(n, 2, 8)
    b = inputs.normal_vector(n, inputs.CG_SEED)
    h = orc.HMatrix(pts, 1, 0.2, 16, 0.0, 1e-8, sigma2=0.1)  # eta=0: H = A
    x, it, rr = orc.HMatrix.cg(h, b, rtol=1e-10, maxit=2000)
    D2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    s = np.sqrt(3 * D2) / 0.2
    A = (1 + s) * np.exp(-s) + 0.1 * np.eye(n)
    xr = np.linalg.solve(A, b)
    assert rr <= 1e-10 and it > 1
    assert _rel(x, xr) <= 1e-8


def test_mlp_forward_special_case(orc):
    # W1 = [I_8; 0], W2 = I_64, W3 = ones, biases 0: yhat = sum_i relu(f_i)
    th = np.zeros(orc.NPARAM)
    W1 = th[:512].reshape(64, 8)
    W1[:8, :8] = np.eye(8)
    W2 = th[576:576 + 4096].reshape(64, 64)
    W2[:] = np.eye(64)
    th[4736:4800] = 1.0
    th[4800] = 0.25
    F = np.random.default_rng(0).standard_normal((10, 8))
    out = orc.mlp_forward(th, F)
    assert np.allclose(out, np.maximum(F, 0).sum(1) + 0.25, rtol=1e-15)


def test_mlp_gradient_finite_differences(orc):
    rng = np.random.default_rng(3)
    th = np.concatenate([
        inputs.he_uniform(8, 64, 1).ravel(), 0.1 * rng.standard_normal(64),
        inputs.he_uniform(64, 64, 2).ravel(), 0.1 * rng.standard_normal(64),
        inputs.he_uniform(64, 1, 3).ravel(), [0.3]])
    assert th.size == orc.NPARAM
    F = rng.standard_normal((20, 8))
    t = rng.standard_normal(20)
    loss, g = orc.mlp_loss_grad(th, F, t)
    idx = rng.choice(orc.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (orc.mlp_loss_grad(tp, F, t)[0] - orc.mlp_loss_grad(tm, F, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_closed_form(orc):
    # after one step from m = v = 0: theta -= lr * g / (|g| + eps)
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    orc.adam_step(th, g, m, v, 1, lr=0.01)
    exp = np.array([1.0, -2.0, 0.5]) - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(th, exp, rtol=1e-12, atol=1e-15)


def _golden_features():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "block_features.txt")
    pts = prm = None
    leaves = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, body = [s.strip() for s in line.split("|", 1)]
        if tag == "points":
            pts = np.array([[float(v) for v in p.split()] for p in body.split(";")])
        elif tag == "params":
            prm = body.split()
        elif tag == "leaf":
            leaves.append([float(v) for v in body.split()])
    return pts, prm, np.array(leaves)


def test_block_features_hand_worked(orc):
    # two hand-placed clusters: diameters, distance and sizes worked out by
    # hand in tests/golden/block_features.txt
    pts, prm, exp = _golden_features()
    leaf, eta, ell, eps, kern = int(prm[0]), float(prm[1]), float(prm[2]), float(prm[3]), int(prm[4])
    O = orc.HMatrix(pts, kern, ell, leaf, eta, eps)
    assert O.n_adm == 2 and O.n_dense == 2
    f = O.features()
    assert f.shape == exp.shape
    assert np.allclose(f, exp, rtol=1e-14, atol=1e-15), (f, exp)


def test_block_features_respond_to_each_input(orc):
    # moving B away by dl in x changes only the distance feature, by
    # log2(1 + (3.375 + dl)/l); a Matern kernel id changes only f7; eps
    # changes only f6
    pts, prm, exp = _golden_features()
    leaf, eta, ell = int(prm[0]), float(prm[1]), float(prm[2])
    p2 = pts.copy()
    p2[2:, 0] += 1.25
    f = orc.HMatrix(p2, 1, ell, leaf, eta, 1e-8).features()
    want = exp.copy()
    want[:, 5] = np.log2(1.0 + (3.375 + 1.25) / ell)
    want[:, 6] = 1.0
    want[:, 7] = 1.0
    assert np.allclose(f, want, rtol=1e-14, atol=1e-15), (f, want)


@pytest.mark.parametrize("steps", [2, 3, 5])
def test_adam_constant_gradient_closed_form(orc, steps):
    # with a constant gradient g from m = v = 0, the bias-corrected moments
    # are exactly m_hat = g and v_hat = g^2 at every step t (the corrections
    # 1 - b^t cancel the geometric sums), so each step moves theta by
    # lr * g / (|g| + eps): a wrong correction exponent at t >= 2 fails here
    th0 = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -4.0, 1e-3, -0.02])
    th, m, v = th0.copy(), np.zeros(4), np.zeros(4)
    for t in range(1, steps + 1):
        orc.adam_step(th, g, m, v, t, lr=0.01)
    exp = th0 - steps * 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(th, exp, rtol=1e-12, atol=1e-15)
    assert np.allclose(m, (1 - 0.9 ** steps) * g, rtol=1e-13)
    assert np.allclose(v, (1 - 0.999 ** steps) * g * g, rtol=1e-12)


def test_adam_sign_flip_second_step(orc):
    # g then -g: m_2 = (0.09 - 0.1) g = -0.01 g, v_2 = (0.000999 + 0.001) g^2;
    # the second step moves against the first by a factor 0.01/0.19 over
    # sqrt(0.001999/0.001999) = 1 relative to |g|, i.e. by lr (1/19) g/|g|
    th0 = np.array([0.7, -1.5])
    g = np.array([2.0, -0.5])
    th, m, v = th0.copy(), np.zeros(2), np.zeros(2)
    orc.adam_step(th, g, m, v, 1, lr=0.1, eps=0.0)
    orc.adam_step(th, -g, m, v, 2, lr=0.1, eps=0.0)
    exp = th0 - 0.1 * np.sign(g) + 0.1 * np.sign(g) / 19.0
    assert np.allclose(th, exp, rtol=1e-13)


def test_oracle_threads_same_factors(orc):
    # the block loops on several threads (used to time the oracle on all
    # host cores): the same ranks and factors, the product to rounding
    pts = inputs.mixture_points(6000, 2, 77)
    x = inputs.normal_vector(6000, 1)
    O = orc.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-7)
    y1 = O.matvec(x)
    r1 = O.ranks()[0].copy()
    U1, V1 = O.factors(len(r1) // 2)
    try:
        orc.set_threads(4)
        O.compress_range(0, O.n_adm)
        y4 = O.matvec(x)
        U4, V4 = O.factors(len(r1) // 2)
    finally:
        orc.set_threads(1)
    assert np.array_equal(O.ranks()[0], r1)
    assert np.array_equal(U1, U4) and np.array_equal(V1, V4)
    assert np.linalg.norm(y4 - y1) <= 1e-14 * np.linalg.norm(y1)

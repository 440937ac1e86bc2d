"""Block-row shares of one H-matrix on the GPU (hm_options row_lo / row_hi).

With the ranges of dist.shard_rows (contiguous Morton rows cut along
cluster-tree nodes, balanced by the product's work), each share's build keeps
only the leaves whose rows meet its range; its product gives the rows of the
range bit for bit as the whole H-matrix does, in FP64, in mixed precision with
the symmetric mode and the rank model, and on the fly. One GPU runs the shares
one after another here; on a node each rank would build one share on its own
GPU and all-gather x (dist.allgather_rows)."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import dist, inputs

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


@pytest.fixture(scope="module")
def theta(hm):
    from paper_1708_09707_gb300 import rank_model
    F, T = rank_model.training_data()
    th, _ = rank_model.train(F, T)
    return th


@pytest.mark.parametrize("mode", ["fp64", "mixed_sym_model", "otf"])
@pytest.mark.parametrize("P", [2, 3])
def test_row_shares_give_the_rows_bit_for_bit(hm, theta, mode, P):
    n = 1 << 15
    pts = inputs.mixture_points(n, 2, 17)
    x = inputs.normal_vector(n, inputs.X_SEED)
    kw = dict(sigma2=0.01)
    if mode == "fp64":
        kw["precision"] = hm.PREC_FP64
    elif mode == "mixed_sym_model":
        kw.update(precision=hm.PREC_MIXED, symmetric=True, rank_model_theta=theta)
    else:
        kw.update(precision=hm.PREC_MIXED, on_the_fly=True)
    H = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, **kw)
    y = H.matvec(x)
    st = H.structure()
    lo, hi, _, _ = H.tree()
    n_adm = H.stats()["n_adm"]
    H.free()
    perm = st["perm"]
    shares = dist.shard_rows(lo, hi, st["adm"], st["dense"], n, P)
    tot_adm = 0
    for r0, r1 in shares:
        Hp = hm.HMatrix(pts, 0, 0.1, 64, 1.0, 1e-6, row_range=(r0, r1), **kw)
        yp = Hp.matvec(x)
        sp = Hp.structure()
        tot_adm += Hp.stats()["n_adm"]
        Hp.free()
        rows = perm[r0:r1]
        assert np.array_equal(yp[rows], y[rows]), (mode, r0, r1)
        assert np.array_equal(sp["perm"], perm)
    # the leaves built twice (row clusters larger than a share) are few
    assert n_adm <= tot_adm <= (1.35 if mode == "mixed_sym_model" else 1.15) * n_adm


def test_row_range_refusals(hm):
    pts = inputs.uniform_points(1000, 2, 3)
    with pytest.raises(hm.HMError):
        hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6, row_range=(10, 5))
    with pytest.raises(hm.HMError):
        hm.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6, row_range=(0, 1001))
    with pytest.raises(hm.HMError):
        hm.HBatch([pts, pts], 0, 0.1, 32, 1.0, 1e-6, row_range=(0, 500))

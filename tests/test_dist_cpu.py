"""The multi-rank path on CPU: two gloo ranks on 127.0.0.1 run the helpers the
bench uses (barrier, max over ranks) and shard a ragged batch of point sets;
every set is owned by exactly one rank and the partition is balanced."""
import os
import socket

import numpy as np
import pytest

from paper_1708_09707_gb300 import dist as hdist
from paper_1708_09707_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        hdist.init("gloo")
        hdist.barrier()
        mx = hdist.max_over_ranks([rank + 1.0, 10.0 * rank, -rank])
        sizes, _ = inputs.ragged_batch_sizes(64, inputs.POINT_SEED + 4)
        mine = hdist.shard_sets(sizes, world, rank)
        hdist.barrier()
        hdist.finalize()
        q.put((rank, mx, mine))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, repr(e), None))


def test_two_gloo_ranks_shard_and_reduce():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, mx, mine = q.get(timeout=120)
        out[rank] = (mx, mine)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] is not None and out[1][1] is not None, out
    assert out[0][0] == out[1][0] == [2.0, 10.0, 0.0]
    sizes, _ = inputs.ragged_batch_sizes(64, inputs.POINT_SEED + 4)
    owned = sorted(out[0][1] + out[1][1])
    assert owned == list(range(64))                    # each set exactly once
    cost = [sum(hdist.set_cost(int(sizes[q])) for q in out[r][1]) for r in range(2)]
    biggest = max(hdist.set_cost(int(s)) for s in sizes)
    assert max(cost) <= sum(cost) / 2 + biggest


def test_shard_sets_single_rank_and_determinism():
    sizes = np.array([5, 100, 7, 100, 3000, 12])
    assert hdist.shard_sets(sizes, 1, 0) == list(range(6))
    a = [hdist.shard_sets(sizes, 3, r) for r in range(3)]
    assert sorted(sum(a, [])) == list(range(6))
    assert a == [hdist.shard_sets(sizes, 3, r) for r in range(3)]
    # the largest set is placed first, alone on rank 0
    assert 4 in a[0]


# ---------------------------------------------------------------------------
# Block-row sharding of one H-matrix (distributed H-matrices, the outlook of
# Sec. 7): ranks own contiguous Morton row ranges; each computes its rows from
# the leaves that touch them after one all-gather of the pieces of x_m.
# ---------------------------------------------------------------------------

def _rows_case(seed=3, n=1 << 13, sym=False):
    import oracle
    pts = inputs.mixture_points(n, 2, seed)
    O = oracle.HMatrix(pts, 0, 0.1, 32, 1.0, 1e-6, symmetric=sym)
    x = inputs.normal_vector(n, inputs.X_SEED)
    return pts, O, x


def _row_worker(rank, world, port, q, sym):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        import torch
        hdist.init("gloo")
        pts, O, x = _rows_case(sym=sym)
        n = pts.shape[0]
        lo, hi, _, _ = O.tree()
        shares = hdist.shard_rows(lo, hi, O.adm_leaves(), O.dense_leaves(), n, world)
        r0, r1 = shares[rank]
        perm = O.perm()
        # this rank holds only its rows' entries of x (in Morton order)
        xm_local = torch.from_numpy(x[perm[r0:r1]].copy())
        xm = hdist.allgather_rows(xm_local, shares).numpy()
        y_local = torch.from_numpy(O.matvec_rows(xm, r0, r1))
        ym = hdist.allgather_rows(y_local, shares).numpy()
        hdist.barrier()
        hdist.finalize()
        y = np.empty(n)
        y[perm] = ym
        q.put((rank, shares, y))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, repr(e), None))


@pytest.mark.parametrize("world,sym", [(2, False), (3, False), (3, True)])
def test_block_row_sharding_gloo(world, sym):
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_row_worker, args=(r, world, port, q, sym)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, shares, y = q.get(timeout=300)
        out[rank] = (shares, y)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(out[r][1] is not None for r in range(world)), out
    _, O, x = _rows_case(sym=sym)
    y_full = O.matvec(x)
    for r in range(world):
        assert out[r][0] == out[0][0]                  # same ranges on every rank
        assert np.array_equal(out[r][1], y_full)       # bit for bit the whole product


def test_shard_rows_partition_properties():
    _, O, x = _rows_case(seed=4, n=1 << 14)
    n = O.n
    lo, hi, _, _ = O.tree()
    A, D = O.adm_leaves(), O.dense_leaves()
    w = hdist.row_work(lo, hi, A, D, n)
    xm = x[O.perm()]
    y_full = O.matvec(x)
    for P in (1, 2, 3, 5, 8):
        sh = hdist.shard_rows(lo, hi, A, D, n, P)
        assert sh[0][0] == 0 and sh[-1][1] == n
        assert all(sh[p][1] == sh[p + 1][0] for p in range(P - 1))
        # every leaf cluster (product tile) lies in one range
        leaves = [v for v in range(len(lo)) if lo[v] >= 0 and
                  (2 * v + 1 >= len(lo) or lo[2 * v + 1] < 0)]
        for v in leaves:
            assert sum(1 for r0, r1 in sh if lo[v] < r1 and hi[v] > r0) == 1
        # balanced to within one candidate node's work of the ideal share
        share = [w[a:b].sum() for a, b in sh]
        assert max(share) <= w.sum() / P * 1.25 + 1e-9, (P, share)
        # the rows of every share are those of the whole product, bit for bit
        ym = np.concatenate([O.matvec_rows(xm, a, b) for a, b in sh])
        y = np.empty(n)
        y[O.perm()] = ym
        assert np.array_equal(y, y_full)
    assert hdist.shard_rows(lo, hi, A, D, n, 1) == [(0, n)]

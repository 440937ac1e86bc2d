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

"""Several GPUs of one node, one process per GPU.

Independent point sets (the batched build, Sec. 4.2 applied across problems)
are spread over the ranks with no data-path collective. One H-matrix is
sharded by block rows (distributed H-matrices, the outlook of Sec. 7): the
Morton-ordered rows are cut into contiguous ranges along cluster-tree nodes,
balanced by the product's work per row (shard_rows); each rank builds only the
leaves whose row cluster meets its range (hm_options row_lo / row_hi) and
computes its rows of every product bit for bit as the whole H-matrix would;
the one exchange per product is an all-gather of the rows' pieces of x (and,
where the caller wants the whole result, of y) (allgather_rows).

Environment: RANK, WORLD_SIZE, LOCAL_RANK and MASTER_ADDR / MASTER_PORT as set
by torch.distributed.run; MASTER_ADDR defaults to 127.0.0.1.
"""
from __future__ import annotations

import math
import os


def world():
    """(world size, rank, local rank) from the environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str, device=None) -> None:
    """Join the process group when there is more than one rank."""
    import torch.distributed as dist
    n, _, _ = world()
    if n > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if device is not None:
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)


def finalize() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def set_cost(n: int) -> float:
    """Work of one point set: the build and the product are O(N log N)."""
    return float(n) * math.log2(max(n, 2))


def shard_sets(sizes, world_size: int, rank: int):
    """Indices of the point sets this rank builds and multiplies.

    Longest-processing-time order: the sets are taken by decreasing cost and
    each goes to the currently least-loaded rank (ties to the lower rank).
    Every set goes to exactly one rank, and no rank carries more than the
    average load plus the largest single set. The result is the same on
    every rank (no communication)."""
    order = sorted(range(len(sizes)), key=lambda q: (-set_cost(int(sizes[q])), q))
    load = [0.0] * world_size
    owner = [0] * len(sizes)
    for q in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        owner[q] = r
        load[r] += set_cost(int(sizes[q]))
    return [q for q in range(len(sizes)) if owner[q] == rank]


def row_work(lo, hi, adm, dense, n: int, kbar: float = 8.0):
    """Work of the product per Morton row: for a dense leaf (tau, sigma) every
    row of tau reads |sigma| near-field entries; for an admissible leaf every
    row reads its k entries of U and a 1/|tau| share of the k |sigma| entries of
    V, with the rank k estimated by kbar. (numpy arrays: node ranges lo, hi;
    leaf lists of node pairs.)"""
    import numpy as np
    diff = np.zeros(n + 1)
    for pairs, dense_leaf in ((adm, False), (dense, True)):
        if len(pairs) == 0:
            continue
        t, s = np.asarray(pairs)[:, 0], np.asarray(pairs)[:, 1]
        m = (hi[t] - lo[t]).astype(np.float64)
        ns = (hi[s] - lo[s]).astype(np.float64)
        w = ns if dense_leaf else kbar * (1.0 + ns / m)
        np.add.at(diff, lo[t], w)
        np.add.at(diff, hi[t], -w)
    return np.cumsum(diff[:n])


def shard_rows(lo, hi, adm, dense, n: int, world_size: int, extra_levels: int = 3,
               kbar: float = 8.0):
    """Block-row ranges [r0, r1) of the Morton order, one per rank.

    The cuts are taken among the first rows of the cluster-tree nodes at depth
    ceil(log2 P) + extra_levels (and of the leaves above that depth), so that
    every leaf cluster lies in one range and only the few leaves whose row
    cluster is larger than a range are built by more than one rank; cut p is
    the candidate whose prefix of row_work is closest to p / P of the total.
    The result depends only on the structure, so every rank computes the same
    ranges without communication. A rank may get an empty range when there are
    fewer candidates than ranks."""
    import numpy as np
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    P = int(world_size)
    if P <= 1:
        return [(0, n)]
    depth = int(math.ceil(math.log2(P))) + extra_levels
    cand = []
    for v in range(len(lo)):
        if lo[v] < 0:
            continue
        dv = int(math.floor(math.log2(v + 1)))
        if dv > depth:
            break
        kids_absent = 2 * v + 1 >= len(lo) or lo[2 * v + 1] < 0
        if dv == depth or kids_absent:
            cand.append(int(lo[v]))
    cand = np.unique(np.asarray([c for c in cand if 0 < c < n], dtype=np.int64))
    w = row_work(lo, hi, adm, dense, n, kbar)
    pref = np.concatenate([[0.0], np.cumsum(w)])
    total = pref[-1]
    cuts = [0]
    for p in range(1, P):
        target = total * p / P
        ok = cand[cand > cuts[-1]]
        if len(ok) == 0:
            cuts.append(cuts[-1])
            continue
        c = int(ok[np.argmin(np.abs(pref[ok] - target))])
        cuts.append(c)
    cuts.append(n)
    return [(cuts[p], max(cuts[p], cuts[p + 1])) for p in range(P)]


def allgather_rows(local, shares):
    """All ranks' row pieces (1-D tensors, rank p holding rows shares[p]) joined
    in rank order on every rank: one all-gather of pieces padded to the
    longest share."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return local.clone()
    width = max(r1 - r0 for r0, r1 in shares)
    pad = torch.zeros(width, dtype=local.dtype, device=local.device)
    pad[: local.numel()] = local
    parts = [torch.empty_like(pad) for _ in shares]
    dist.all_gather(parts, pad)
    return torch.cat([parts[p][: r1 - r0] for p, (r0, r1) in enumerate(shares)])

"""Several GPUs of one node, one process per GPU.

The H-matrix path shards without a data-path collective. Independent point
sets (the batched build, Sec. 4.2 applied across problems) are spread over
the ranks, and a single point set runs as replicas. Only scalars such as
timings cross ranks. Block-row sharding of one H-matrix with an all-gather of
x is not built.

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

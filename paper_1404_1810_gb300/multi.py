"""Work sharing across GPUs, one process per GPU.

The transforms of a batch are independent (the DFT of Eq. qft_0A of each one
needs only its own samples), so ranks exchange nothing on the data path: a
batch is split into contiguous shards, a ragged list of lengths is
partitioned by its cost N log2 N, and only timings are reduced (the maximum
over ranks, the job's wall time).
"""
from __future__ import annotations

import heapq


def shard(total: int, world: int, rank: int) -> tuple[int, int]:
    """(first, count) of rank's contiguous share of `total` transforms; the
    first total % world ranks take one more."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def partition_ragged(log2n, world: int) -> list:
    """Indices of a ragged list for each rank, balancing sum(N log2 N):
    longest-processing-time first onto the least loaded rank (ties to the
    lowest rank), each rank's indices in increasing order."""
    import numpy as np

    lg = np.asarray(log2n, dtype=np.int64)
    cost = (np.int64(1) << lg) * np.maximum(lg, 1)
    order = np.lexsort((np.arange(len(lg)), -cost))   # by cost, descending; stable
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + int(cost[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def max_over_ranks(value: float) -> float:
    """The maximum of `value` over the ranks of the default process group
    (the value itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Host-side logic of multi-process runs: one process per GPU, independent graphs per rank.

Ordering one graph does not shard (its level-synchronous traversal would need a per-level
exchange between GPUs, the paper's distributed design of Sec. IV), so several GPUs run independent
replicas or independent graphs: no collective touches the data path. The only collectives are the
timing reductions below.
"""
from __future__ import annotations

import heapq


def shard_by_size(sizes, world: int) -> list[list[int]]:
    """Partition graph indices over `world` ranks, balancing the total size per rank (greedy:
    largest graph first, to the least-loaded rank; ties to the lower rank). Every index appears in
    exactly one shard; indices keep their increasing order inside a shard."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(s) for s in shards]


def assemble(parts, count: int) -> list:
    """Per-graph results of all ranks back in the original order: parts holds one mapping
    {graph index: result} per rank (each rank ordered its shard). Raises if a graph is missing or
    was returned by more than one rank."""
    out = [None] * count
    seen = [False] * count
    for part in parts:
        for i, res in part.items():
            if not 0 <= i < count:
                raise ValueError(f"graph index {i} outside the batch of {count}")
            if seen[i]:
                raise ValueError(f"graph {i} returned by more than one rank")
            seen[i] = True
            out[i] = res
    missing = [i for i in range(count) if not seen[i]]
    if missing:
        raise ValueError(f"{len(missing)} graphs returned by no rank, first {missing[:5]}")
    return out


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job takes as long as its slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """The sum of `value` over all ranks (units processed by the whole job)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

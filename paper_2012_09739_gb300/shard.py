"""Sharding a level estimate across ranks (one process per GPU).

Samples are independent and their random numbers are a function of the path
index alone (counter-based generator), so rank r of W simulates the
contiguous range of paths given by shard_range and nothing is exchanged
until the sums: one all-reduce of (sum D, sum D^2, n) per level and
estimator yields exactly the samples of a single-GPU run over the whole
range (up to the order of the final additions).
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int, offset: int = 0) -> tuple[int, int]:
    """(path_offset, count) of this rank's share of paths offset .. offset+n-1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return offset + start, count


def allreduce_sums(s1: float, s2: float, n: int, group=None) -> tuple[float, float, int]:
    """Sums over all ranks (torch.distributed, any backend; FP64)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([s1, s2, float(n)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t[0]), float(t[1]), int(round(float(t[2])))


def max_over_ranks(x: float, group=None) -> float:
    """Maximum of a per-rank value (the timing rule of the benchmark)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t[0])

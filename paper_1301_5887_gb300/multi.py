"""Multi-GPU helpers for the sampling stage (host side, torch.distributed).

The CSR build does not shard (each GPU holds a replica of the graph), but the
samples do: every stream's index range [0, k) is cut into contiguous shards
(`shard_range`), each rank draws its shard with `first_sample`, and one
integer all-reduce (sum) of the counter block (`allreduce_counts`) gives
exactly the counts one GPU would produce, because samples are keyed by
their index. `max_over_ranks` reduces per-rank step times for timing.
Works with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import numpy as np

STAT_BINS = 34


def shard_range(k: int, rank: int, world: int):
    """(first, count) of rank's contiguous share of sample indices [0, k)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(int(k), world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def counter_block(counts_matrix, k_global: int, closed_global: int, stats) -> np.ndarray:
    """Flatten (n_bins x 5 tallies, global pair, statistics) into one int64 block."""
    cm = np.asarray(counts_matrix, dtype=np.uint64).reshape(-1)
    st = np.asarray(stats, dtype=np.uint64).reshape(-1)
    return np.concatenate([cm, np.array([k_global, closed_global], np.uint64), st]).view(np.int64)


def split_block(block: np.ndarray, n_bins: int):
    b = np.asarray(block, dtype=np.int64).view(np.uint64)
    cm = b[: n_bins * 5].reshape(n_bins, 5)
    kg, cg = int(b[n_bins * 5]), int(b[n_bins * 5 + 1])
    stats = b[n_bins * 5 + 2:].reshape(STAT_BINS, STAT_BINS)
    return cm, kg, cg, stats


def allreduce_counts(counts_matrix, k_global: int, closed_global: int, stats, group=None):
    """Sum the integer counter blocks of all ranks (exact). Returns
    (counts_matrix, k_global, closed_global, stats)."""
    import torch
    import torch.distributed as dist
    block = counter_block(counts_matrix, k_global, closed_global, stats)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.as_tensor(block.copy(), device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return split_block(t.cpu().numpy(), np.asarray(counts_matrix).shape[0])


def max_over_ranks(x: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

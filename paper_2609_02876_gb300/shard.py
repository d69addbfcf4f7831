"""Trajectory sharding across ranks (one process per GPU).

Trajectories are independent (paper Sec. 3.1), so an ensemble splits into
contiguous ranges with no exchange; the gradients of each rank's trajectories
are final on that rank. The only cross-rank reduction of the path is the LV
UDE's shared-weight gradient (a sum over all trajectories): it is gathered
and added in rank order in FP64, so every rank obtains the same bits
whatever the process layout.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of the trajectories owned by `rank`: contiguous, sizes differ by at most one."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def sum_in_rank_order(parts) -> np.ndarray:
    """The shards' shared-weight gradients added one after another in shard (rank)
    order, in FP64: the reduction every rank performs on the gathered vectors."""
    acc = np.zeros(np.asarray(parts[0]).shape, dtype=np.float64)
    for p in parts:
        acc += np.asarray(p, dtype=np.float64)
    return acc


def sum_shared_grad(local: np.ndarray, group=None) -> np.ndarray:
    """Deterministic all-reduce of a shared-weight gradient: every rank's vector is
    gathered and the vectors are added in rank order in FP64."""
    t = torch.as_tensor(np.ascontiguousarray(local, dtype=np.float64))
    if not dist.is_available() or not dist.is_initialized():
        return t.numpy().copy()
    world = dist.get_world_size(group)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    return sum_in_rank_order([q.numpy() for q in parts])


def max_over_ranks(x: float, group=None, device=None) -> float:
    """Maximum of a scalar over all ranks (the timing rule of the benchmark)."""
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

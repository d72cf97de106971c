"""Replica sharding for several GPUs (one process per GPU).

Samples are independent, so N GPUs run N replicas of the single-GPU path on disjoint
seed ranges; no collective touches the data path.  The only exchanges are host-level:
the timing maximum of a benchmark step and, for estimators, gathering per-sample
results back into seed order.  torch.distributed is the transport (NCCL on GPUs, gloo
on CPU).
"""
from typing import Tuple

import numpy as np


def shard(total: int, world: int, rank: int) -> Tuple[int, int]:
    """[start, stop) of rank's share of `total` samples (contiguous, sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_in_order(local: np.ndarray, total: int, world: int, rank: int, group=None) -> np.ndarray:
    """All ranks' per-sample values back in global seed order (every rank gets all)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return np.asarray(local, dtype=np.float64)
    start, stop = shard(total, world, rank)
    buf = torch.zeros(total, dtype=torch.float64)
    buf[start:stop] = torch.as_tensor(np.asarray(local, dtype=np.float64))
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = buf.to(dev)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)  # disjoint supports: the sum is a gather
    return buf.cpu().numpy()


def max_over_ranks(x: float, world: int, group=None) -> float:
    import torch
    import torch.distributed as dist
    if world == 1:
        return float(x)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

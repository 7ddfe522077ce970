"""Multi-GPU host logic: one process per GPU, cells sharded across ranks with no
exchange of lattice data (Couette cells are independent problems), timings
combined as the maximum over ranks, per-cell results gathered on rank 0.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple

import numpy as np


def rank_world() -> Tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (0, 1, 0 alone)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world %d/%d" % (rank, world))
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over all ranks (the job's wall time is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local: np.ndarray, n_items: int, device=None) -> np.ndarray:
    """Concatenates per-rank blocks (rows = items in shard order) on every rank."""
    import torch
    import torch.distributed as dist
    local = np.ascontiguousarray(local, dtype=np.float64)
    if not (dist.is_available() and dist.is_initialized()):
        return local
    world = dist.get_world_size()
    width = local.shape[1] if local.ndim == 2 else 1
    sizes = [len(shard(n_items, r, world)) for r in range(world)]
    m = max(sizes)
    buf = torch.zeros((m, width), dtype=torch.float64, device=device)
    buf[: local.shape[0]] = torch.from_numpy(local.reshape(-1, width)).to(buf.device)
    out = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(out, buf)
    rows: List[np.ndarray] = [o[:s].cpu().numpy() for o, s in zip(out, sizes)]
    res = np.concatenate(rows, axis=0)
    return res if local.ndim == 2 else res[:, 0]


def job_rate(units_per_rank: Sequence[float], seconds_max: float) -> float:
    """Whole-job throughput: units processed by all ranks / the slowest rank's time."""
    return float(sum(units_per_rank)) / float(seconds_max)

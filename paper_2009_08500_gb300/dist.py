"""Multi-process helpers (one process per GPU, launched by torchrun).

The light-curve path needs no data exchange: every (parameter vector,
time) is independent, so a batch of parameter vectors is split across
ranks and each rank evaluates its share on its own GPU.  The only
collectives are for measurement: a barrier around the timed region and the
maximum of the per-rank times.
"""
from __future__ import annotations

import os
from typing import Tuple


def env() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous share [lo, hi) of n items for `rank`; sizes differ by at most one."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def init(backend: str = "nccl") -> None:
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (the value itself with one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

"""Multi-GPU bookkeeping of the detection path (one process per GPU).

The path shards with no data-path collective: every rank analyses its own
strain (its own hour, segments or streams).  The only collectives are the
timing barrier and the reduction of the per-rank results: the job's time is
the slowest rank's, and the job's throughput is the units all ranks
processed divided by that time (weak scaling).
"""
from __future__ import annotations

import os
from typing import Tuple


def env() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank r's synthetic strain (rank 0 keeps the single-GPU workload)."""
    return base_seed + 7919 * rank


def job_throughput(local_units: float, local_seconds: float, world: int = 1) -> Tuple[float, float, float]:
    """(units/s of the whole job, total units, job seconds): units summed over
    ranks, time = max over ranks.  Collective when world > 1."""
    if world <= 1:
        return local_units / local_seconds, local_units, local_seconds
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(u.item()), float(t.item())


def barrier(world: int = 1) -> None:
    """All ranks meet (when world > 1), then this rank's device is idle."""
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()

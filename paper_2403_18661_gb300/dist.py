"""Multi-GPU bookkeeping of the detection path (one process per GPU).

Two ways to use several GPUs, both without a collective inside the path:
* independent work per rank (its own hour, segments or streams): the only
  collectives are the timing barrier and the reduction of the per-rank
  results (weak scaling);
* one timeslide background split across ranks (Sec. IX: the background is
  the union of many timeslides of the same strain): every rank whitens the
  same segments and takes a contiguous range of the timeslides
  (shift_range), then the ranks exchange their background triggers once
  (gather_background, kilobytes per rank) so that every rank can assign
  false-alarm rates against the whole background (strong scaling).
The job's time is the slowest rank's, and the job's throughput is the units
all ranks processed divided by that time.
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


def shift_range(n_shift: int, world: int, rank: int) -> Tuple[int, int]:
    """(first timeslide k, count) of rank `rank` when timeslides k = 1 .. n_shift are split into
    `world` contiguous ranges whose sizes differ by at most one (earlier ranks take the extra)."""
    if n_shift < world:
        raise ValueError(f"{n_shift} timeslides cannot be split over {world} ranks")
    base, extra = divmod(n_shift, world)
    count = base + (1 if rank < extra else 0)
    first = 1 + rank * base + min(rank, extra)
    return first, count


def gather_background(values, world: int = 1):
    """Concatenate every rank's background statistics (1-D float32 tensor, on the device of the
    process group's backend), in rank order, on every rank.  Two collectives: the counts, then
    the values padded to the largest count."""
    if world <= 1:
        return values
    import torch
    import torch.distributed as dist
    n = torch.tensor([values.numel()], dtype=torch.int64, device=values.device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    m = max(max(counts), 1)
    padded = torch.zeros(m, dtype=values.dtype, device=values.device)
    padded[: values.numel()] = values
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])


def sum_over_ranks(x: float, world: int = 1) -> float:
    """Sum of a per-rank number (e.g. the background livetime of each rank's timeslides)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

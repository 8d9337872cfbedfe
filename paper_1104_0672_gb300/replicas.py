"""Host logic of the multi-GPU form: independent replicas, one process per GPU.

Maps are independent problems, so N GPUs run N replicas with their own batches and no
collective on the data path.  The only collectives are host-side bookkeeping: a barrier
around the timed region and the maximum of the per-rank step times (the slowest rank bounds
the job), from which the whole-job throughput is formed.  Launched by torchrun, which sets
RANK / LOCAL_RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT.
"""
from __future__ import annotations

import os


def env():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 when absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world: int, backend: str):
    """The process group for world > 1 (None for a single process)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist


def map_config(rank: int, base: int = 3) -> int:
    """Seed configuration of a rank's synthetic maps: every replica convolves different maps."""
    return base + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pixels_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job Gpix*maps/s: the pixels every rank convolves per step over the slowest rank's
    step time."""
    return pixels_per_rank * world / (ms_per_step * 1e-3) / 1e9

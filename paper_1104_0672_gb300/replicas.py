"""Host logic of the multi-GPU form: independent replicas, one process per GPU.

Maps are independent problems, so N GPUs run N replicas with their own batches and no
collective on the forward data path.  The collectives are host-side bookkeeping -- a barrier
around the timed region and the maximum of the per-rank step times (the slowest rank bounds
the job), from which the whole-job throughput is formed -- and, when the ranks fit one beam
shared by all their maps, the sum of the per-rank knot gradients after each backward pass
(allreduce_knot_grad): the loss is a sum over maps, so its gradient with respect to the shared
knots is the sum of every rank's gradient over its own maps.  Launched by torchrun, which sets
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


def allreduce_knot_grad(grad_knots, dist=None, group=None):
    """Sum, in place, a shared beam's knot gradient [nkernels, T] over all ranks (the gradient
    of the summed loss of every rank's maps); returns it.  FP64 on any device the process
    group's backend takes (gloo: CPU; NCCL: CUDA).  Without a process group it is returned
    unchanged."""
    if dist is None:
        return grad_knots
    dist.all_reduce(grad_knots, op=dist.ReduceOp.SUM, group=group)
    return grad_knots

"""Replica bookkeeping for running independent solves on several GPUs.

The constraint solve has no exchange step between problems: each rank solves its
own instances with its own context, and the only collective is the timing
reduction below (a barrier and a max of the wall time), which is not on the data
path.  Works with any ``torch.distributed`` backend (NCCL on GPUs, gloo on CPU).
"""
import os


def dist_env():
    """(world_size, rank, local_rank) from the torchrun environment; (1, 0, 0) without it."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(secs, device="cpu"):
    """Slowest rank's time.  Every rank calls it; returns ``secs`` when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(secs)
    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(units_per_rank, secs_max, world_size):
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    if secs_max <= 0:
        raise ValueError("non-positive timing")
    return world_size * units_per_rank / secs_max

"""Replica bookkeeping for runs on several GPUs of one node.

The benchmark's multi-GPU mode runs one independent copy of the problem per
rank (the loss and gradient of separate reconstructions share no data), so
the only cross-rank work is timing: every rank times its own steps and the
job's time is the slowest rank's.  These helpers work with any initialised
torch.distributed process group (NCCL on GPUs, gloo on CPU for tests).
"""
import torch
import torch.distributed as dist


def world():
    """(rank, world size) of the current process group, (0, 1) without one."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def max_over_ranks(value, device="cpu"):
    """The maximum of `value` (a float) over all ranks."""
    rank, size = world()
    if size == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step, steps, world_size, slowest_ms):
    """Units processed by all ranks per second of the slowest rank."""
    if slowest_ms <= 0:
        raise ValueError("non-positive time")
    return units_per_step * steps * world_size / (slowest_ms / 1e3)

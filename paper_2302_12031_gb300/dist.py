"""Multi-process helpers: one process per GPU, replicas of the same work.

The trace has no exchange step between GPUs in this build: every rank traces
its own full problem (replicas), so the only cross-rank operations are a
barrier around the timed region and the maximum of the ranks' times. They run
on any torch.distributed backend (NCCL on GPUs, gloo on CPUs for tests).
"""
import os

import torch
import torch.distributed as dist


def env():
    """(rank, world_size, local_rank) from the torchrun environment (0, 1, 0 without it)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend):
    """Join the process group when launched with more than one rank."""
    rank, world, _ = env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return rank, world


def barrier(device=None):
    if dist.is_available() and dist.is_initialized():
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()
    if device is not None and device.type == "cuda":
        torch.cuda.synchronize(device)


def max_over_ranks(value, device=None):
    """The largest `value` (a float) over all ranks; the value itself with one rank."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    if device is None:   # NCCL reduces device tensors only
        device = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, seconds_per_rank, device=None):
    """Whole-job throughput of replicas: all ranks' units over the slowest rank's time."""
    world = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    t = max_over_ranks(seconds_per_rank, device)
    return world * units_per_rank / t, t

"""Runs on several GPUs of one node, one process per GPU (launched by
torchrun).  The frames are independent, so the ranks share nothing on the
data path (replicas): each rank extracts its own frame, and only the timing
is combined -- the slowest rank's time, and a whole-job rate that counts
every rank's pixels.  The functions work on any torch.distributed backend
(NCCL on GPUs, gloo on CPUs for the host-side tests)."""
from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) from the torchrun environment."""
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def init(world: int, backend: str = "nccl", device=None):
    """The process group when world > 1 (else None)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=device)
    else:
        dist.init_process_group(backend)
    return dist


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist, device="cpu") -> float:
    """The largest value of x over the ranks (every rank gets it)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def frame_seed(rank: int) -> int:
    """Seed of the rank's frame: independent frames, one per rank."""
    return rank


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / seconds


def finish(dist) -> None:
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()

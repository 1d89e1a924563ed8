"""Replica runs across ranks: one process per GPU, each advancing its own copy
of the workload (a single mesh is not partitioned; no exchange happens on the
data path). These host helpers read the launcher's environment, reduce a
per-rank time to the slowest rank's and turn it into the whole job's rate."""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the default process group (x itself
    without one); `device` holds the reduction tensor (a CUDA device under
    NCCL, the CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms_per_step: float, world_size: int) -> float:
    """Units per second of the whole job: every rank's units of one step over
    the slowest rank's step time."""
    return world_size * units_per_rank / (ms_per_step * 1e-3)

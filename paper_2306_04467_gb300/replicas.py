"""Runs across ranks, one process per GPU, with no exchange on the data path.

A single mesh is not partitioned: each rank advances its own replica. An
ensemble of independent instances is sharded: each rank advances a subset of
the instances (balanced by triangle count) and only the per-instance
statistics meet on the host at the end. These helpers read the launcher's
environment, split the instances, reduce a per-rank time to the slowest
rank's, gather per-instance results and turn units and time into the whole
job's rate."""
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


def partition_instances(sizes, world_size: int):
    """Split instances of the given triangle counts over world_size ranks:
    largest first, each to the rank with the fewest triangles so far (ties to
    the lower rank); returns each rank's instance indices in ascending order.
    Deterministic, so every rank computes the same split."""
    load = [0] * world_size
    parts = [[] for _ in range(world_size)]
    for i in sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(p) for p in parts]


def gather_instance_results(local: dict, n_instances: int):
    """Per-instance results (instance index -> list of floats) of every rank,
    merged into one list in instance order on every rank (the host-side
    exchange at the end of a sharded run; the local dict itself without a
    process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, local)
    else:
        parts = [local]
    merged = {}
    for p in parts:
        for k, v in p.items():
            if int(k) in merged:
                raise ValueError("instance %d reported by two ranks" % int(k))
            merged[int(k)] = v
    if sorted(merged) != list(range(n_instances)):
        raise ValueError("instances missing from the gathered results")
    return [merged[i] for i in range(n_instances)]

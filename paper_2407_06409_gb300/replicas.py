"""Whole-job throughput of independent replicas (one structure per GPU, no data exchange).

The local-cluster problems of different structures share nothing, so N GPUs run N
independent structures.  The job time is the slowest rank's time and the work is the sum
of every rank's atoms; the reduction runs over whatever torch.distributed process group is
initialised (NCCL on GPUs, gloo in the CPU tests), or is the identity without one.
"""
from __future__ import annotations


def job_throughput(local_seconds: float, local_units: float, device=None) -> tuple[float, float]:
    """(max seconds over ranks, sum of units over ranks / max seconds)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_seconds), float(local_units) / float(local_seconds)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item()) / float(t.item())

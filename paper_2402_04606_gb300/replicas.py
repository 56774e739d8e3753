"""Replicas on several GPUs: independent instances per rank, no data-path
collective.  The only cross-rank step is the timing reduction of a
benchmark: the whole job's rate is the units all ranks processed over the
slowest rank's time."""
from __future__ import annotations


def max_over_ranks(value: float) -> float:
    """The maximum of ``value`` over the ranks of the default process group
    (the value itself without one, or with a single rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, slowest_seconds: float, world: int) -> float:
    """Whole-job throughput of ``world`` replicas that each processed
    ``units_per_rank`` units, timed by the slowest rank."""
    return world * units_per_rank / slowest_seconds

"""Host logic of multi-GPU runs: every rank generates the corrections of its own copy of
the workload (independent surfaces shard with no exchange on the data path), and the
job's time is that of the slowest rank."""
from __future__ import annotations


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over the ranks of the default process group (the value itself
    without one).  `device`: where the reduction tensor lives (a CUDA device under NCCL,
    the CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank: int, steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job points/s of a weak-scaling run: all ranks' points over the slowest rank's
    time."""
    return world * points_per_rank * steps / (slowest_ms / 1e3)

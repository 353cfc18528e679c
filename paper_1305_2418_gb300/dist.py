"""Multi-process helpers of the benchmark: every rank solves its own replica
(the solves are independent; there is no collective on the data path).  The
only collectives are the timing barrier and two reductions of the results:
the step time is the max over ranks and the update counts are summed."""
from __future__ import annotations

import os


def env():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(local_units: float, local_ms: float, device=None) -> tuple[float, float]:
    """(units of all ranks per second, max step time over ranks in ms)."""
    ms = max_over_ranks(local_ms, device)
    return sum_over_ranks(local_units, device) / (ms / 1e3), ms

"""Independent replicas across ranks (one GPU each, no data-path collective).

The solver does not shard a grid across GPUs: each rank runs its own solves.
Timing follows the usual rule: every rank's elapsed time is reduced with MAX
(the job takes as long as its slowest rank) and the work with SUM.
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(elapsed: float, units: float, device=None):
    """(max elapsed over ranks, total units over ranks); a no-op on one rank.
    device: where the reduction tensors live (cuda for NCCL, cpu for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed), float(units)
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())

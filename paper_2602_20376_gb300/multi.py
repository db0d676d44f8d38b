"""Multi-GPU plumbing of the sampling path: candidates are independent, so
ranks score disjoint direction streams against a replicated V and exchange
only their winners (Sec. 5: no communication between workers until the best
candidate is returned).

* ``direction_seed``: the seed of step s on rank g (disjoint streams).
* ``merge_best``: all-gather of each rank's (f, candidate index) and the
  global winner (largest f; ties to the lower rank, then the lower index).
* ``max_over_ranks``: the job's time is the slowest rank's.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def direction_seed(step: int, world: int, rank: int) -> int:
    return 1 + step * world + rank


def merge_best(best_f: float, best_idx: int, device="cpu"):
    """Returns (f, rank, idx) of the global winner; every rank gets the same."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(best_f), 0, int(best_idx)
    world = dist.get_world_size()
    mine = torch.tensor([float(best_f), float(dist.get_rank()), float(best_idx)], dtype=torch.float64,
                        device=device)
    allv = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(allv, mine)
    rows = sorted(((-float(t[0]), int(t[1]), int(t[2])) for t in allv))
    f, rank, idx = rows[0]
    return -f, rank, idx


def max_over_ranks(value: float, device="cpu") -> float:
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Several GPUs: independent populations, one per rank.

The method's runs are independent, so N GPUs run N independent populations (rank r uses seed
base + r) with no collective on the data path; only the measurement needs the ranks: the
slowest rank's time and the total work.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def rank_seed(base_seed: int, rank: int) -> int:
    return int(base_seed) + int(rank)


def aggregate(ms: float, sweep_ms: float, attempts: float, device: torch.device | str = "cpu"):
    """(max over ranks of ms, max of sweep_ms, sum of attempts); identity without a process
    group.  `device` is where the reduction tensor lives (cpu for gloo, cuda for nccl)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(sweep_ms), float(attempts)
    t = torch.tensor([ms, sweep_ms], dtype=torch.float64, device=device)
    a = torch.tensor([attempts], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), float(a[0])

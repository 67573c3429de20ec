"""Replica runs on several GPUs of one node (one process per GPU).

Each rank advances its own copy of the workload (the hot path needs no
collective on one mesh); the whole-job throughput is the work of all ranks
divided by the slowest rank's time.  This module holds only that host logic
so that it can be tested with the gloo backend on CPU.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier() -> None:
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device: str = "cpu") -> float:
    """Largest value of x over all ranks (the slowest rank's time)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device: str = "cpu") -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_local: float, seconds_local: float, device: str = "cpu") -> float:
    """Units processed by all ranks / the slowest rank's time (weak scaling:
    every rank does the same fixed amount of work)."""
    return sum_over_ranks(units_local, device) / max_over_ranks(seconds_local, device)

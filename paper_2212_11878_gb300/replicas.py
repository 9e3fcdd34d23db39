"""Host logic of the multi-GPU replica runs: one process per GPU, each advancing its own
independent box (the single-box SRD step has no exchange step once a box fits one GPU).

Ranks differ only in their seeds; the job's throughput is the updates of all ranks divided
by the slowest rank's time.  Works on any torch.distributed backend (NCCL on GPUs, gloo
on CPU ranks in the tests).
"""
from __future__ import annotations


def box_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s replica of a single box."""
    return int(seed) + int(rank)


def ensemble_seed(seed: int, rank: int) -> int:
    """Seed of one box of rank `rank`'s replica of an ensemble (boxes keep distinct seeds)."""
    return int(seed) + 1000003 * int(rank)


def job_throughput(local_updates: float, local_ms: float, dist=None, device=None):
    """(updates per second of the whole job, slowest rank's ms, total updates).  Without an
    initialised process group this is the single-process value."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_updates / (local_ms / 1e3), local_ms, local_updates
    import torch
    ms = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    upd = torch.tensor([float(local_updates)], dtype=torch.float64, device=device)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(upd, op=dist.ReduceOp.SUM)
    ms_max, total = float(ms.item()), float(upd.item())
    return total / (ms_max / 1e3), ms_max, total

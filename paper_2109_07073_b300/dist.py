"""Multi-process plumbing for running independent replicas of the workload.

Factors, overlap pairs and voxelmaps are independent units, so N processes (one
per GPU) each process their own batch; nothing is exchanged on the data path.
Only the timing needs the ranks: a barrier on both sides of the timed region
and the maximum step time over ranks.
"""
from __future__ import annotations

import os


def rank_world():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def init(backend: str = "nccl"):
    """Join the process group named by the launcher's environment (no-op for one rank)."""
    rank, world = rank_world()
    if world > 1:
        import torch.distributed as tdist
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        if not tdist.is_initialized():
            tdist.init_process_group(backend)
    return rank, world


def barrier(world: int):
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the slowest rank's step time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, world: int, ms_per_step_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's step time."""
    return units_per_rank * world / (ms_per_step_max / 1e3)

"""Multi-process plumbing for running the level advance on several GPUs of
one node: one process per GPU, each advancing its own meshes.

Meshes are independent problems, so ranks exchange no data while they
step: each rank runs its own copy of the workload (weak scaling), and the
only collectives are the barrier around the timed region and two scalar
reductions afterwards -- the slowest rank's time and the total work.
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init(backend: str, device=None) -> None:
    import torch.distributed as dist
    if device is not None and backend == "nccl":
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)


def _reduce(x: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "max", device)


def sum_over_ranks(x: float, device=None) -> float:
    return _reduce(x, "sum", device)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()


def finalize() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()
        dist.destroy_process_group()


def throughput(units_local: float, seconds_local: float, device=None) -> tuple[float, float]:
    """Whole-job rate: the units every rank processed over the slowest
    rank's time.  Returns (rate, slowest time)."""
    t = max_over_ranks(seconds_local, device)
    u = sum_over_ranks(units_local, device)
    return u / t, t

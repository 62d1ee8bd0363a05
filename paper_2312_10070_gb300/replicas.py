"""Host-side logic of multi-GPU runs.

The rasterizer's mapping and tracking steps of one keyframe exchange no data,
so an N-GPU run is N independent replicas, one process per GPU: every rank
times its own steps and the whole-job figure is the units all ranks processed
over the slowest rank's time.  These helpers are backend-agnostic (NCCL on
GPUs, gloo on CPU in the tests).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> int:
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def _device():
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(x: float) -> float:
    """The maximum of x over all ranks (x itself in a single process)."""
    if world() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    if world() > 1:
        dist.barrier()


def whole_job_rate(units_per_rank: float, local_seconds: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return world() * units_per_rank / max_over_ranks(local_seconds)

"""Whole-job throughput of independent replicas (one lattice per rank).

The method's hot path has no exchange step when runs are independent, so a
multi-GPU job here is N replicas: every rank advances its own lattice and the job's
throughput is the units of all ranks divided by the slowest rank's time. The only
collectives are these two host-side reductions (no data-path communication).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def job_throughput(local_seconds: float, local_units: float, device=None):
    """Return (units of all ranks / max seconds over ranks, max seconds, total units).

    Works without torch.distributed (a single process) and with any backend; pass a
    CUDA device for NCCL, None (CPU) for gloo."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local_units / local_seconds, local_seconds, local_units
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    secs, units = float(t.item()), float(u.item())
    return units / secs, secs, units

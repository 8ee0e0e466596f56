"""Host-side coordination of independent replicas (one process per GPU).

ECB blocks are independent (paper abstract: every 64-bit block is encrypted
on its own), so several GPUs simply run separate buffers: there is no data
exchange at all.  The ranks only agree on timing: a barrier before and after
the timed region, the slowest rank's time, and the sum of the work.  A rank
that fails or never arrives is detected by a barrier with a deadline instead
of a hang.
"""
from __future__ import annotations

import datetime


def world():
    """(rank, world_size) from torch.distributed, or (0, 1) when not initialised."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def barrier(timeout_s: float | None = None) -> None:
    """Barrier across ranks.  With a timeout (gloo), a rank that does not
    arrive in time makes the others raise RuntimeError naming it."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return
    if timeout_s is not None and dist.get_backend() == "gloo":
        dist.monitored_barrier(timeout=datetime.timedelta(seconds=timeout_s))
    else:
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gbs(bytes_per_rank: int, max_ms: float, world_size: int) -> float:
    """Whole-job throughput: every rank's bytes over the slowest rank's time."""
    return bytes_per_rank * world_size / (max_ms * 1e-3) / 1e9

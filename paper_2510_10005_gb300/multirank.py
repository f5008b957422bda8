"""Host-side logic of multi-GPU jobs: one process per GPU under
torch.distributed (NCCL on GPUs, gloo in the CPU tests).

Cells are independent (the chemistry of a cell never reads another cell), so
a job gives every rank its own block of cells and moves nothing between
ranks on the data path. The collectives are bookkeeping: the job's time is
the slowest rank's, its throughput counts the cells of all ranks, and the
adjoint's parameter gradient (a sum over cells) is summed over ranks once.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_total: int, world: int, rank: int):
    """Contiguous block [start, stop) of rank out of n_total cells; block
    sizes differ by at most one cell."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def barrier():
    d = _dist()
    if d is not None:
        d.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over ranks (the job's time is its slowest rank's)."""
    d = _dist()
    if d is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks_(t):
    """In-place sum over ranks of a tensor (the adjoint's dL/dtheta)."""
    d = _dist()
    if d is not None:
        d.all_reduce(t)
    return t


def job_throughput(cells_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Cells of the whole job per second, weak scaling: every rank holds
    cells_per_rank cells and the time is the slowest rank's."""
    return world * cells_per_rank * steps / seconds

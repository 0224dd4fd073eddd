"""Multi-GPU host logic: one process per GPU, lines of sight are independent.

RM synthesis has no exchange step (every LOS is its own contraction, Sec. 3),
so the only collectives are bookkeeping: a barrier around the timed region and
the maximum of the ranks' times.  Work is either replicated per rank (weak
scaling: each rank synthesises a cube of its own) or a contiguous LOS range per
rank (strong scaling of one cube).
"""
from __future__ import annotations


def los_range(nlos: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [start, stop) of rank's lines of sight; sizes differ by at most 1."""
    if world < 1 or not 0 <= rank < world or nlos < 0:
        raise ValueError("bad rank/world/nlos")
    base, extra = divmod(nlos, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(t_ms: float, device=None) -> float:
    """The largest value of t_ms over all ranks (all_reduce MAX); t_ms itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_ms)
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: int, steps: int, t_ms_local: float, world: int, device=None):
    """(whole-job units per second / 1e9, slowest rank's ms): all ranks' units over the slowest rank's time."""
    tmax = max_over_ranks(t_ms_local, device)
    return world * units_per_rank * steps / (tmax * 1e-3) / 1e9, tmax

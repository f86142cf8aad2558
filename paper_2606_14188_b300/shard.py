"""Multi-GPU layout of the path: rollouts and served requests are independent, so ranks take
disjoint shares with no collective on the data path; the only collectives are the benchmark's
barrier and its max-over-ranks of the timed interval.  Host logic only (no kernels)."""
from __future__ import annotations


def rollout_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share [lo, hi) of `total` rollouts for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def route(request_index: int, world: int) -> int:
    """Rank that serves a plan request: requests go whole to one GPU, round-robin by arrival."""
    return request_index % world


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over the ranks of the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

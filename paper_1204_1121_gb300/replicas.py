"""Replica-parallel host logic (one process per GPU, no data-path collective).

Walkers are independent, so every rank holds the whole coefficient table and
evaluates its own walkers.  Two ways to give ranks their walkers:

* weak scaling: every rank gets a full workload of its own (distinct position
  streams), so the work per GPU is fixed as ranks are added;
* strong scaling: the walkers of one workload are split into contiguous,
  near-equal ranges.

The only collective is the reduction of the step time (maximum over ranks),
which is timing, not data.
"""
from __future__ import annotations


def walker_range(n_walkers: int, rank: int, world: int):
    """Contiguous walker range [w0, w1) of ``rank`` for strong scaling."""
    if world < 1 or not (0 <= rank < world) or n_walkers < 0:
        raise ValueError("bad rank/world/walker count")
    return (n_walkers * rank) // world, (n_walkers * (rank + 1)) // world


def weak_seed(base_seed: int, rank: int) -> int:
    """Position-stream seed of ``rank`` for weak scaling (distinct per rank)."""
    return base_seed + 1000 * rank


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of a per-rank scalar (e.g. ms per step) over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    x = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(x, op=dist.ReduceOp.MAX, group=group)
    return float(x.item())

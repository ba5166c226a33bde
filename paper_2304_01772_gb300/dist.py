"""Multi-GPU sharding of independent lattice batches (one process per GPU).

Lattices never exchange data during sweeps, so N GPUs run N independent
batches (weak scaling): rank r runs the full batch with seed `seed + r`.
Throughput is the units processed on all ranks divided by the slowest rank's
time; that max over ranks is taken after the timed region.  The one exchange
of the method is the gradient over chains that share theta but live on
different GPUs: an all-reduce (sum) of the pooled integer moments, carried
as 32-bit limbs so that the sum is exact (`pooled_gradient`).
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world, local_rank) from the torchrun environment (single process: 0, 1, 0)."""
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", rank))
    return rank, world, local


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`: distinct Philox keys, so the ranks' chains are independent."""
    return (seed + rank) & ((1 << 64) - 1)


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over all ranks (the slowest rank's time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate: units processed on all ranks / slowest rank's time."""
    return units_per_rank * world / seconds


def allreduce_limbs(limbs, dist=None):
    """Element-wise SUM of limb tensors over ranks, in place (exact: int64
    sums of 32-bit limbs)."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(limbs, op=dist.ReduceOp.SUM)
    return limbs


def pooled_gradient(sim, first, n, observable=0, dist=None):
    """Gradient and expectations pooled over the chains of all ranks: each rank
    pools its lattices' moments into limbs, the limbs are summed over ranks, and
    the library forms the estimator from the sum."""
    limbs = sim.pooled_limbs(first, n)
    allreduce_limbs(limbs, dist)
    return sim.grad_from_limbs(limbs, observable)


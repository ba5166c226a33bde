"""Multi-GPU sharding of a lattice batch (one process per GPU).

Lattices never exchange data during sweeps, so the batch axis is the natural
shard (the paper's batch dimension B of its [B, C, H, W] tensor, Sec.
"Methods"): `partition_by_sites` splits one batch over the ranks by site count
(greedy largest-first bin packing of the ragged sizes), and `rank_lattices`
gives each rank its lattices with lattice_id = global index + 1, so that every
lattice draws the Philox numbers it would draw in the whole batch and the
ranks together run exactly the one-GPU chains (strong scaling, no data-path
collective).  The weak-scaling alternative gives every rank the whole batch
under its own seed (`rank_seed`).  Throughput is the units processed on all
ranks divided by the slowest rank's time; that max over ranks is taken after
the timed region.  The one exchange of the method is the gradient over chains
that share theta but live on different GPUs: an all-reduce (sum) of the pooled
integer moments, carried as 32-bit limbs so that the sum is exact
(`pooled_gradient`).
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world, local_rank) from the torchrun environment (single process: 0, 1, 0)."""
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", rank))
    return rank, world, local


def partition_by_sites(sizes, world: int):
    """Split lattices of sides `sizes` over `world` ranks by site count: the
    lattices in decreasing L^2 (ties by index) each go to the rank with the
    fewest sites so far (ties to the lowest rank).  Deterministic: every rank
    computes the same split.  Returns one ascending list of lattice indices
    per rank; no rank's load exceeds the mean by more than the largest lattice."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 2, i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += int(sizes[i]) ** 2
    return [sorted(p) for p in parts]


def rank_lattices(lattices, rank: int, world: int):
    """This rank's share of a batch: (lattice dicts with lattice_id = global
    index + 1, their global indices)."""
    idx = partition_by_sites([d["L"] for d in lattices], world)[rank]
    return [dict(lattices[i], lattice_id=i + 1) for i in idx], idx


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank` in the weak-scaling mode (every rank runs the whole
    batch): distinct Philox keys, so the ranks' chains are independent."""
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


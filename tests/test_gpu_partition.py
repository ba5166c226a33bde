"""A batch split over several contexts reproduces the batch in one context.

The batch axis is the multi-GPU shard: paper_2304_01772_gb300.dist splits a
batch over ranks by site count and gives every lattice lattice_id = global
index + 1, so each lattice draws the numbers it draws in the whole batch.
Here two contexts on one GPU stand for two ranks: together they must give the
one-context spins and per-sweep statistics bit for bit (initial state
included), in the launch forms a rank would use."""
import numpy as np
import pytest
import torch

import paper_2304_01772_gb300 as sm
from paper_2304_01772_gb300 import dist as sdist
from paper_2304_01772_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SEED = 0x5A5A12345


@pytest.mark.parametrize("world,form", [(2, (0, True, 0, 512)), (3, (0, True, 0, 256)), (2, (1, True, 0, 256))])
def test_split_batch_reproduces_the_whole_batch(world, form):
    lats = wl.uneven512(n=60, seed=11, emin=4, emax=11)     # 16 .. 2048: tile and strip kernels
    whole = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=8)
    whole.set_launch(*form)
    init_whole = whole.spins.cpu().numpy().copy()
    whole.sweep(6, record=True)
    st_whole = whole.observables_host(0, 6)[0]
    parts = []
    for r in range(world):
        mine, idx = sdist.rank_lattices(lats, r, world)
        sim = sm.Sim(sm.SPIN_ISING, mine, seed=SEED, max_record=8)
        sim.set_launch(*form)
        for k, gi in enumerate(idx):          # the same random start
            L = lats[gi]["L"]
            a = init_whole[whole.offsets[gi]:whole.offsets[gi] + L * L]
            assert np.array_equal(sim.lattice(k).cpu().numpy().ravel(), a), (r, gi)
        sim.sweep(6, record=True)
        parts.append((sim, idx, sim.observables_host(0, 6)[0]))
    seen = []
    for sim, idx, st in parts:
        for k, gi in enumerate(idx):
            assert torch.equal(sim.lattice(k), whole.lattice(gi)), gi
            assert np.array_equal(st[:, k], st_whole[:, gi]), gi
        seen += idx
    assert sorted(seen) == list(range(len(lats)))


def test_lattice_id_defaults_to_the_batch_index():
    lats = wl.uneven512(n=6, seed=2, emin=4, emax=8)
    a = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=4)
    b = sm.Sim(sm.SPIN_ISING, [dict(d, lattice_id=i + 1) for i, d in enumerate(lats)], seed=SEED, max_record=4)
    c = sm.Sim(sm.SPIN_ISING, [dict(d, lattice_id=len(lats) - i) for i, d in enumerate(lats)], seed=SEED,
               max_record=4)
    for s in (a, b, c):
        s.sweep(3, record=True)
    assert torch.equal(a.spins, b.spins)
    assert np.array_equal(a.observables_host(0, 3)[0], b.observables_host(0, 3)[0])
    assert not torch.equal(a.spins, c.spins)    # other words, other chains

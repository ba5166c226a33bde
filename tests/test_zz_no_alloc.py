"""The allocation-free Ising sweep (spin_ising_sweep_noalloc) against the
context-based sweep (spin_init / spin_sweep).

spin_ising_sweep_noalloc exists for callers that cannot call cudaMalloc (code
inside another framework's memory pool or allocator hook, processes whose
device memory is reserved up front); it keeps its scratch in a fixed static
device array instead.  Both paths run the same chain, so spins and the
per-sweep statistics must agree exactly -- here over two calls in a row, the
second continuing the chain where the first stopped.
"""
import ctypes

import pytest
import torch

import paper_2304_01772_gb300 as sm

pytestmark = pytest.mark.gpu

SEED = 0x00C0FFEE12345678
LATS = [dict(L=4, beta=0.3, J=1.0, h=0.0), dict(L=10, beta=0.44, J=-1.0, h=0.1),
        dict(L=16, beta=0.2, J=1.0, h=0.05), dict(L=48, beta=0.6, J=0.7, h=-0.2),
        dict(L=64, beta=0.44, J=1.0, h=0.0), dict(L=128, beta=0.35, J=1.0, h=0.01),
        dict(L=256, beta=0.5, J=1.0, h=0.0), dict(L=512, beta=0.41, J=1.0, h=-0.03)]


def _descs(lats, offsets):
    arr = (sm.LatticeDesc * len(lats))()
    for i, d in enumerate(lats):
        arr[i] = sm.LatticeDesc(d["L"], 2, d["beta"], d["J"], d["h"], 0, 0.0, 0, offsets[i])
    return arr


def _noalloc(desc, n, spins, first, count, stats):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return sm.lib().spin_ising_sweep_noalloc(ctypes.c_uint64(SEED), n, desc, spins.data_ptr(), first,
                                             count, stats.data_ptr() if stats is not None else None,
                                             stream)


def test_noalloc_matches_context_sweep_over_two_calls():
    n = len(LATS)
    sim = sm.Sim(sm.SPIN_ISING, LATS, seed=SEED, max_record=16)
    spins = sim.spins.clone()                      # the same random start
    desc = _descs(LATS, sim.offsets)
    first_stats = torch.full((5, n, 2), -7, dtype=torch.int64, device="cuda")
    assert _noalloc(desc, n, spins, 0, 5, first_stats) == 0
    sim.sweep(5, record=True)
    torch.cuda.synchronize()
    assert torch.equal(spins, sim.spins)
    assert torch.equal(first_stats, sim.observables(0, 5)[0])
    second_stats = torch.full((3, n, 2), -7, dtype=torch.int64, device="cuda")
    assert _noalloc(desc, n, spins, 5, 3, second_stats) == 0
    sim.sweep(3, record=True)
    torch.cuda.synchronize()
    assert torch.equal(spins, sim.spins)
    assert torch.equal(second_stats, sim.observables(5, 3)[0])


def test_noalloc_rejects_odd_sides():
    spins = torch.zeros(16, dtype=torch.int8, device="cuda")   # never touched: rejected first
    odd = [dict(L=7, beta=0.4, J=1.0, h=0.0)]
    assert _noalloc(_descs(odd, [0]), 1, spins, 0, 1, None) == -1


def test_noalloc_near_its_scratch_limit_matches_context_and_oracle():
    """Three 2048^2 lattices (12 MiB of the 16 MiB scratch with their second
    buffer) next to small ones: the allocation-free call runs them on the tile
    kernel, the context on the row-strip kernel; both give the oracle's chain."""
    import numpy as np

    import oracle
    lats = [dict(L=2048, beta=0.44, J=1.0, h=0.0), dict(L=32, beta=0.3, J=1.0, h=0.1),
            dict(L=2048, beta=0.5, J=1.0, h=-0.02), dict(L=10, beta=0.4, J=-1.0, h=0.0),
            dict(L=2048, beta=0.3, J=0.8, h=0.05)]
    n = len(lats)
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=8)
    assert max(o + d["L"] ** 2 for o, d in zip(sim.offsets, lats)) > 12 * 2 ** 20
    spins = sim.spins.clone()
    init = {i: sim.lattice(i).cpu().numpy().copy() for i in (0, 1, 3)}
    desc = _descs(lats, sim.offsets)
    stats = torch.full((2, n, 2), -7, dtype=torch.int64, device="cuda")
    assert _noalloc(desc, n, spins, 0, 2, stats) == 0
    sim.sweep(2, record=True)
    torch.cuda.synchronize()
    assert torch.equal(spins, sim.spins)
    assert torch.equal(stats, sim.observables(0, 2)[0])
    for i, s0 in init.items():
        d = lats[i]
        ref = oracle.ising_run(s0, d["beta"], d["J"], d["h"], SEED, i, 0, 2)
        L = d["L"]
        got = spins[sim.offsets[i]:sim.offsets[i] + L * L].view(L, L).cpu().numpy()
        assert np.array_equal(got, s0), i
        assert np.array_equal(stats[:, i].cpu().numpy(), ref), i


def test_noalloc_rejects_a_span_beyond_its_scratch_and_sides_above_2048():
    # four 2048^2 lattices pass every per-lattice check, but their span (16 MiB)
    # plus the descriptors cannot fit in the 16 MiB array
    lats = [dict(L=2048, beta=0.4, J=1.0, h=0.0)] * 4
    spins = torch.zeros(16, dtype=torch.int8, device="cuda")   # never touched: rejected first
    assert _noalloc(_descs(lats, [k * 2048 * 2048 for k in range(4)]), 4, spins, 0, 1, None) == -1
    big = [dict(L=4096, beta=0.4, J=1.0, h=0.0)]
    assert _noalloc(_descs(big, [0]), 1, spins, 0, 1, None) == -1

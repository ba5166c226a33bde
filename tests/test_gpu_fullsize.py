"""GPU parity at the benchmark's full sizes, in the launch forms it times.

The uneven Ising batch (512 lattices, L = 2^e, e in 5..11) runs in the form
the autotuner picks for the benchmark: work lists of 8-warp strip blocks with
balanced row ranges, replayed from a captured graph.  50 sweeps are compared
with the oracle from the random start: integer statistics after every sweep,
spins after sweeps 1, 10 and 50, on every lattice up to 256^2 and one lattice
of each larger side.  The Potts batches (64 lattices of 1024^2, q = 3 and 8)
run in the autotuner's form and are compared on three lattices the same way.

The oracle runs in a thread pool (its C entry points release the GIL), so no
process is forked after the GPU is in use.
"""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2304_01772_gb300 as sm
from paper_2304_01772_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SEED = 0xC0FFEE12345
CHECKPOINTS = (1, 10, 50)


def _host_lattices(sim, idx):
    flat = sim.spins.cpu().numpy()
    return {i: flat[sim.offsets[i]:sim.offsets[i] + sim.sizes[i] ** 2].reshape(sim.sizes[i], sim.sizes[i]).copy()
            for i in idx}


def _pool():
    return ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)))


def _ising_sample(lats):
    seen, idx = set(), []
    for i, d in enumerate(lats):
        if d["L"] <= 256 or d["L"] not in seen:
            seen.add(d["L"])
            idx.append(i)
    return idx


def test_uneven512_benchmark_form_50_sweeps():
    lats = wl.uneven512()
    idx = _ising_sample(lats)
    assert {lats[i]["L"] for i in idx} == {32, 64, 128, 256, 512, 1024, 2048}
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=64)
    sim.set_launch(0, True, 0, 512)
    assert sim.get_launch() == {"mode": 0, "use_graph": 1, "tile_rows": 0, "threads": 512}
    ref = _host_lattices(sim, idx)
    got_spins, t = {}, 0
    for k in CHECKPOINTS:
        sim.sweep(k - t, record=True)
        t = k
        got_spins[k] = _host_lattices(sim, idx)
    st = sim.observables_host(0, CHECKPOINTS[-1])[0]

    def run(i):
        d, s = lats[i], ref[i]
        out, stats, t0 = {}, [], 0
        for k in CHECKPOINTS:
            stats.append(oracle.ising_run(s, d["beta"], d["J"], d["h"], SEED, i, t0, k - t0))
            out[k] = s.copy()
            t0 = k
        return i, out, np.concatenate(stats)

    with _pool() as ex:
        for i, out, stats in ex.map(run, idx):
            for k in CHECKPOINTS:
                assert np.array_equal(got_spins[k][i], out[k]), (i, lats[i]["L"], k)
            assert np.array_equal(st[:, i, :], stats), (i, lats[i]["L"])
    # the running statistics equal the last record
    assert torch.equal(sim.observables(CHECKPOINTS[-1] - 1, 1)[0][0], sim.current_stats())


@pytest.mark.parametrize("q", [3, 8])
def test_potts_batch_benchmark_form_50_sweeps(q):
    lats = wl.potts_batch(q)
    pick = [0, 37, 63]
    sim = sm.Sim(sm.SPIN_POTTS, lats, seed=SEED, max_record=64)
    sim.autotune(4)          # the form the benchmark times (the state is restored)
    ref = _host_lattices(sim, pick)
    got_spins, t = {}, 0
    for k in CHECKPOINTS:
        sim.sweep(k - t, record=True)
        t = k
        got_spins[k] = _host_lattices(sim, pick)
    st = sim.observables_host(0, CHECKPOINTS[-1])[0]

    def run(i):
        d, s = lats[i], ref[i]
        out, stats, t0 = {}, [], 0
        for k in CHECKPOINTS:
            stats.append(oracle.potts_run(s, q, d["beta"], d["J"], SEED, i, t0, k - t0))
            out[k] = s.copy()
            t0 = k
        return i, out, np.concatenate(stats)

    with _pool() as ex:
        for i, out, stats in ex.map(run, pick):
            for k in CHECKPOINTS:
                assert np.array_equal(got_spins[k][i], out[k]), (i, k, sim.get_launch())
            assert np.array_equal(st[:, i, :], stats), (i, sim.get_launch())

"""GPU parity of the Ising path with first and second neighbours (geometry 2,
Sec. "Ising model": the checkerboard update with four colours) against the
CPU oracle: spins bit for bit after every sweep, the statistics (M, B, B2)
exactly, E and M per site to FP32 rounding, the fluctuation estimator of
d<O>/d(J, h, J2) to 1e-9 relative, in every launch form (per-colour kernels
batched or in place, with and without graphs, and the resident form)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import estimator
import paper_2304_01772_gb300 as sm
from paper_2304_01772_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SEED = 0x5EED1234ABCD

# sides cover L/2 not a multiple of 4 (Philox groups crossing rows), a ragged
# tail of groups, one-block and many-block lattices
NNN = [dict(L=L, beta=b, J=J, J2=J2, h=h, geometry=2) for L, b, J, J2, h in [
    (4, 0.3, 1.0, 0.5, 0.0), (6, 0.4, 1.0, -0.5, 0.1), (10, 0.35, -1.0, 0.3, -0.05),
    (16, 0.3, 1.0, -0.25, 0.0), (30, 0.45, 1.0, 0.4, 0.02), (64, 0.2, 0.5, -0.5, 0.0),
    (130, 0.3, 1.0, 0.1, -0.1), (256, 0.28, 1.0, -0.4, 0.0)]]


def f32(v):
    return float(np.float32(v))


def lattice_np(sim, i):
    return sim.lattice(i).cpu().numpy().copy()


def check_chain(sim, lats, init, t0, n, first, idx=None):
    st, E, M = sim.observables_host(first, n)
    for i in (range(len(lats)) if idx is None else idx):
        d = lats[i]
        s = init[i].copy()
        ref = oracle.nnn_run(s, d["beta"], d["J"], d["J2"], d["h"], SEED, i, t0, n)
        assert np.array_equal(lattice_np(sim, i), s), (i, d)
        assert np.array_equal(st[:, i, :], ref), (i, d)
        N = d["L"] ** 2
        e = (-f32(d["J"]) * ref[:, 1] - f32(d["J2"]) * ref[:, 2] - f32(d["h"]) * ref[:, 0]) / N
        np.testing.assert_allclose(E[:, i], e.astype(np.float32), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(M[:, i], (ref[:, 0] / N).astype(np.float32), rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("mode,graph", [(0, True), (0, False), (1, False), (1, True), (2, True), (2, False)])
def test_second_neighbour_sweeps_match_the_oracle(mode, graph):
    lats = NNN + ([dict(L=512, beta=0.3, J=1.0, J2=-0.2, h=0.0, geometry=2)] if mode != 2 else [])
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=16)
    assert sim.width == 3
    sim.set_launch(mode, graph, 0, 512 if mode == 2 else 256)
    init = {i: lattice_np(sim, i) for i in range(len(lats))}
    st0 = sim.current_stats().cpu().numpy()
    for i, d in enumerate(lats):
        assert np.array_equal(init[i], oracle.init_ising(d["L"], SEED, i)), i
        assert np.array_equal(st0[i], oracle.nnn_stats(init[i])), i
    sim.sweep(1, record=True)
    sim.sweep(4, record=True)   # odd count: the batched form ends with a copy back
    check_chain(sim, lats, init, 0, 5, 0)
    assert np.array_equal(sim.current_stats().cpu().numpy(), sim.observables_host(4, 1)[0][0])


@pytest.mark.parametrize("form", ["batched", "resident", "tuned"])
def test_second_neighbour_benchmark_workload_sampled(form):
    """The benchmark's 256 lattices of 256^2 in the launch form the benchmark
    picks (autotuned) and in both fixed forms; lattices sampled for the oracle."""
    lats = wl.nnn256()
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=4)
    if form == "tuned":
        sim.autotune(2)
    else:
        sim.set_launch(0 if form == "batched" else 2, True, 0, 512)
    pick = [0, 77, 200, 255]
    init = {i: lattice_np(sim, i) for i in pick}
    sim.sweep(3, record=True)
    check_chain(sim, lats, init, 0, 3, 0, idx=pick)


def test_second_neighbour_gradient_matches_the_oracle_estimator():
    b, J, J2, h = 0.3, 1.0, -0.4, 0.05
    lats = [dict(L=32, beta=b, J=J, J2=J2, h=h, geometry=2) for _ in range(4)]
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=400)
    sim.sweep(300, record=True)
    st = sim.observables_host(0, 300)[0]          # [T, n_lat, 3]
    args = (f32(b), f32(J), f32(J2), f32(h), 32 * 32)
    for obs, name in [(0, "E"), (1, "M")]:
        g = sim.grad(100, 200, observable=obs).cpu().numpy()
        gp = sim.grad(100, 200, observable=obs, pool=True).cpu().numpy()
        assert g.shape == (4, 3)
        for i in range(4):
            ref = estimator.nnn_grad(st[100:, i][None], *args)
            want = [ref[(name, "J")], ref[(name, "h")], ref[(name, "J2")]]
            np.testing.assert_allclose(g[i], want, rtol=1e-9, atol=1e-12)
        refp = estimator.nnn_grad(np.transpose(st[100:], (1, 0, 2)), *args)
        np.testing.assert_allclose(gp[0], [refp[(name, "J")], refp[(name, "h")], refp[(name, "J2")]],
                                   rtol=1e-9, atol=1e-12)
    ex = sim.expectations(100, 200).cpu().numpy()
    for i in range(4):
        X = st[100:, i].astype(np.float64)
        E = (-f32(J) * X[:, 1] - f32(J2) * X[:, 2] - f32(h) * X[:, 0]) / 1024
        np.testing.assert_allclose(ex[i], [E.mean(), X[:, 0].mean() / 1024], rtol=1e-12, atol=1e-15)


def test_second_neighbour_load_checkpoint_and_restore():
    lats = NNN[:6]
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=8)
    sim.sweep(3, record=True)
    torch.cuda.synchronize()
    kept = sim.current_stats().clone()
    span = int(sim.spins.numel())
    host = torch.zeros(span, dtype=torch.int8).pin_memory()
    sim.store_spins(host)
    sim.load_spins(host)
    torch.cuda.synchronize()
    assert torch.equal(sim.current_stats(), kept)
    rng = np.random.default_rng(5)
    new = torch.from_numpy(rng.choice(np.array([-1, 1], dtype=np.int8), size=span)).pin_memory()
    sim.load_spins(new)
    torch.cuda.synchronize()
    init = {i: lattice_np(sim, i) for i in range(len(lats))}
    cur = sim.current_stats().cpu().numpy()
    for i in range(len(lats)):
        assert np.array_equal(cur[i], oracle.nnn_stats(init[i])), i
    blob = sim.checkpoint()
    first = sim.n_records
    sim.sweep(2, record=True)
    check_chain(sim, lats, init, 3, 2, first)
    after = {i: lattice_np(sim, i) for i in range(len(lats))}
    sim.restore(blob)
    sim.sweep(2, record=True)
    for i in range(len(lats)):
        assert np.array_equal(lattice_np(sim, i), after[i]), i

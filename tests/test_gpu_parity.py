"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Spin configurations must match bit for bit after every sweep, integer
statistics exactly, and FP32 observables to within 1e-6 relative (they are
formed in double from the same integers and rounded once, so in practice
they are equal).  Lattices are independent, so full-size batches are checked
by running the oracle on a sample of their lattices.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_01772_gb300 as sm
from paper_2304_01772_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SEED = 0x5EED1234ABCD


def lattice_np(sim, i):
    return sim.lattice(i).cpu().numpy().copy()


def oracle_ising_chain(lats, seed, init, t0, n, idx=None):
    """Run the oracle on lattices `idx` (their batch indices) from `init`."""
    idx = range(len(lats)) if idx is None else idx
    out, stats = {}, {}
    for i in idx:
        d = lats[i]
        s = init[i].copy()
        stats[i] = oracle.ising_run(s, d["beta"], d["J"], d["h"], seed, i, t0, n)
        out[i] = s
    return out, stats


def make_ising(lats, seed=SEED, max_record=64, **kw):
    return sm.Sim(sm.SPIN_ISING, lats, seed=seed, max_record=max_record, **kw)


MIXED = [dict(L=L, beta=b, J=J, h=h) for L, b, J, h in [
    (4, 0.3, 1.0, 0.0), (6, 0.5, -1.0, 0.1), (10, 0.44, 1.0, -0.2), (16, 0.2, 1.0, 0.05),
    (32, 0.6, 1.0, 0.0), (48, 0.44, 0.7, 0.3), (64, 0.35, 1.0, -0.05), (128, 0.44, 1.0, 0.0),
    (144, 0.5, 1.0, 0.02), (256, 0.41, 1.0, 0.0), (12, 0.0, 1.0, 0.0), (96, 3.0, 1.0, 0.0)]]


def test_init_matches_oracle():
    sim = make_ising(MIXED)
    for i, d in enumerate(MIXED):
        assert np.array_equal(lattice_np(sim, i), oracle.init_ising(d["L"], SEED, i))
    st = sim.current_stats().cpu().numpy()
    for i in range(len(MIXED)):
        assert list(st[i]) == list(oracle.ising_stats(lattice_np(sim, i)))


@pytest.mark.parametrize("mode,graph,tile,threads", [(0, False, 0, 256), (0, True, 0, 256),
                                                     (0, True, 8, 128), (0, False, 64, 512),
                                                     (1, False, 0, 256), (1, True, 0, 256),
                                                     (3, True, 0, 512), (3, False, 16, 256)])
def test_ising_mixed_batch_sweep_by_sweep(mode, graph, tile, threads):
    sim = make_ising(MIXED)
    sim.set_launch(mode, graph, tile, threads)
    init = {i: lattice_np(sim, i) for i in range(len(MIXED))}
    ref = {i: init[i].copy() for i in init}
    for t in range(4):
        sim.sweep(1, record=True)
        for i, d in enumerate(MIXED):
            oracle.ising_sweep(ref[i], d["beta"], d["J"], d["h"], SEED, i, t)
            assert np.array_equal(lattice_np(sim, i), ref[i]), (t, i, d)
    # longer stretch in one call (graph replay + odd remainder), then compare
    sim.sweep(7, record=True)
    got_st, E, M = sim.observables_host(0, 11)
    for i, d in enumerate(MIXED):
        st = oracle.ising_run(ref[i], d["beta"], d["J"], d["h"], SEED, i, 4, 7)
        assert np.array_equal(lattice_np(sim, i), ref[i])
        assert np.array_equal(got_st[4:, i, :], st)
        N = d["L"] ** 2
        Eo = (-float(np.float32(d["J"])) * st[:, 1] - float(np.float32(d["h"])) * st[:, 0]) / N
        np.testing.assert_allclose(E[4:, i], Eo.astype(np.float32), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(M[4:, i], (st[:, 0] / N).astype(np.float32), rtol=1e-6, atol=1e-7)
    assert sim.t == 11 and sim.n_records == 11


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_resident_form_matches_oracle_and_batched(threads):
    lats = [dict(L=L, beta=b, J=J, h=h) for L, b, J, h in [
        (16, 0.3, 1.0, 0.0), (32, 0.44, 1.0, 0.1), (64, 0.6, -1.0, 0.0), (128, 0.4, 0.8, -0.05),
        (256, 0.5, 1.0, 0.02), (64, 0.2, 1.0, 0.0)]]
    sim = make_ising(lats, max_record=32)
    sim.set_launch(2, False, 0, threads)
    ref = {i: lattice_np(sim, i) for i in range(len(lats))}
    for t in range(2):
        sim.sweep(1, record=True)
        for i, d in enumerate(lats):
            oracle.ising_sweep(ref[i], d["beta"], d["J"], d["h"], SEED, i, t)
            assert np.array_equal(lattice_np(sim, i), ref[i]), (t, i)
    sim.sweep(9, record=True)
    st = sim.observables_host(0, 11)[0]
    for i, d in enumerate(lats):
        o = oracle.ising_run(ref[i], d["beta"], d["J"], d["h"], SEED, i, 2, 9)
        assert np.array_equal(lattice_np(sim, i), ref[i])
        assert np.array_equal(st[2:, i], o)
    other = make_ising(lats, max_record=32)
    other.sweep(11, record=True)
    assert torch.equal(other.spins, sim.spins)
    assert np.array_equal(other.observables_host(0, 11)[0], st)
    assert torch.equal(sim.current_stats(), sim.observables(10, 1)[0][0])


@pytest.mark.parametrize("cs,threads", [(2, 256), (2, 1024), (4, 512), (4, 1024)])
def test_resident_cluster_form_matches_oracle(cs, threads):
    """Each lattice split over a cluster of cs CTAs (rows exchanged through
    distributed shared memory): bit-identical to the oracle sweep by sweep,
    over calls of several sweeps, and to the one-CTA resident form."""
    lats = [dict(L=L, beta=b, J=J, h=h) for L, b, J, h in [
        (16, 0.3, 1.0, 0.0), (32, 0.44, 1.0, 0.1), (64, 0.6, -1.0, 0.0), (128, 0.4, 0.8, -0.05),
        (256, 0.5, 1.0, 0.02), (64, 0.2, 1.0, 0.0), (256, 0.44, 1.0, 0.0)]]
    sim = make_ising(lats, max_record=32)
    sim.set_launch(2, False, cs, threads)
    assert sim.get_launch() == {"mode": 2, "use_graph": 0, "tile_rows": cs, "threads": threads}
    ref = {i: lattice_np(sim, i) for i in range(len(lats))}
    for t in range(2):
        sim.sweep(1, record=True)
        for i, d in enumerate(lats):
            oracle.ising_sweep(ref[i], d["beta"], d["J"], d["h"], SEED, i, t)
            assert np.array_equal(lattice_np(sim, i), ref[i]), (t, i)
    sim.sweep(3, record=True)
    sim.sweep(6, record=True)
    st = sim.observables_host(0, 11)[0]
    for i, d in enumerate(lats):
        o = oracle.ising_run(ref[i], d["beta"], d["J"], d["h"], SEED, i, 2, 9)
        assert np.array_equal(lattice_np(sim, i), ref[i]), i
        assert np.array_equal(st[2:, i], o), i
    other = make_ising(lats, max_record=32)
    other.set_launch(2, True, -1, 512)
    other.sweep(11, record=True)
    assert torch.equal(other.spins, sim.spins)
    assert np.array_equal(other.observables_host(0, 11)[0], st)
    assert torch.equal(sim.current_stats(), sim.observables(10, 1)[0][0])


def test_resident_cluster_form_in_a_graph_and_back():
    """The cluster form replayed from a graph, then the batched form, continue one chain."""
    lats = wl.fit256(n=6, L=256) + [dict(L=128, beta=0.3, J=1.0, h=0.1)]
    a, b = make_ising(lats), make_ising(lats)
    a.set_launch(2, True, 4, 1024)
    a.sweep(5, record=True)
    a.set_launch(0, True, -1, 512)
    a.sweep(3, record=True)
    b.sweep(8, record=True)
    assert torch.equal(a.spins, b.spins)
    assert np.array_equal(a.observables_host(0, 8)[0], b.observables_host(0, 8)[0])


def test_launch_forms_bit_identical():
    lats = wl.uneven512(n=40, seed=3, emin=4, emax=9)
    finals = []
    for mode, graph, tile, threads in [(0, True, 0, 256), (0, False, 16, 128), (1, True, 0, 256),
                                       (0, True, 64, 512), (3, True, 0, 512), (3, False, 0, 256)]:
        sim = make_ising(lats, max_record=16)
        sim.set_launch(mode, graph, tile, threads)
        sim.sweep(9, record=True)
        st, E, M = sim.observables(0, 9)
        finals.append((sim.spins.cpu().numpy(), st.cpu().numpy()))
        sim.close()
    for s, st in finals[1:]:
        assert np.array_equal(s, finals[0][0])
        assert np.array_equal(st, finals[0][1])


@pytest.mark.parametrize("rows,warps", [(0, 256), (1, 256), (5, 128), (7, 256), (32, 128)])
def test_strip_kernel_rows_and_tail(rows, warps):
    """Lattices of side 512, 1024 and 2048 take the warp row-strip kernel; item
    heights that are not multiples of the 4-step unroll exercise its tail."""
    lats = [dict(L=512, beta=0.44, J=1.0, h=0.03), dict(L=1024, beta=0.3, J=1.0, h=-0.1),
            dict(L=2048, beta=0.5, J=-0.8, h=0.0), dict(L=64, beta=0.4, J=1.0, h=0.0)]
    sim = make_ising(lats, max_record=8)
    sim.set_launch(0, True, rows, warps)
    init = [lattice_np(sim, i) for i in range(len(lats))]
    sim.sweep(3, record=True)
    st = sim.observables_host(0, 3)[0]
    for i, d in enumerate(lats):
        ref = oracle.ising_run(init[i], d["beta"], d["J"], d["h"], SEED, i, 0, 3)
        assert np.array_equal(lattice_np(sim, i), init[i]), i
        assert np.array_equal(st[:, i, :], ref), i


@pytest.mark.parametrize("mode,graph,threads", [(0, True, 512), (0, False, 256), (3, True, 512), (3, False, 512)])
def test_split_rows_between_the_sweeps_of_a_call(mode, graph, threads):
    """Within one call of n sweeps the strip lattices stay in the strip kernel's
    split row form between sweeps (the first sweep reads and the last one
    writes int8 rows): every sweep count per call, with and without graphs,
    continues the oracle's chain, and the state is int8 after each call."""
    lats = [dict(L=512, beta=0.44, J=1.0, h=0.03), dict(L=1024, beta=0.35, J=1.0, h=-0.05),
            dict(L=64, beta=0.4, J=1.0, h=0.0)]
    sim = make_ising(lats, max_record=32)
    sim.set_launch(mode, graph, 0, threads)
    ref = [lattice_np(sim, i) for i in range(len(lats))]
    t = 0
    for n in (1, 2, 3, 4, 5):
        sim.sweep(n, record=True)
        st = sim.observables_host(t, n)[0]
        for i, d in enumerate(lats):
            exp = oracle.ising_run(ref[i], d["beta"], d["J"], d["h"], SEED, i, t, n)
            assert np.array_equal(lattice_np(sim, i), ref[i]), (n, i)
            assert np.array_equal(st[:, i, :], exp), (n, i)
        t += n


def test_contexts_with_different_shared_memory_needs_coexist():
    """A context planned later with smaller work items must not lower the
    shared-memory limit that an earlier context's launches rely on."""
    big = make_ising([dict(L=256, beta=0.44, J=1.0, h=0.0)], max_record=4)
    big.set_launch(0, False, 200, 256)          # (200 + 4) * 256 B > 48 KB of shared memory
    small = make_ising([dict(L=32, beta=0.44, J=1.0, h=0.0)], max_record=4)
    small.sweep(1)
    s0 = lattice_np(big, 0)
    big.sweep(1)
    oracle.ising_sweep(s0, 0.44, 1.0, 0.0, SEED, 0, 0)
    assert np.array_equal(lattice_np(big, 0), s0)


def test_autotune_picks_a_form_and_keeps_results(tmp_path, monkeypatch):
    lats = wl.uneven512(n=24, seed=11, emin=5, emax=10)
    ref = make_ising(lats, max_record=8)
    ref.sweep(6, record=True)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SPINMC_TUNE_CACHE", str(cache))
    sim = make_ising(lats, max_record=8)
    choice = sim.autotune(sweeps_per_trial=2)
    assert choice["mode"] in (0, 1) and choice["threads"] in (128, 256, 512)
    assert sim.t == 0 and sim.n_records == 0          # trials leave the chain where it was
    sim.sweep(6, record=True)
    assert torch.equal(sim.spins, ref.spins)
    assert np.array_equal(sim.observables_host()[0], ref.observables_host()[0])
    # the choice is cached per batch shape and reused without timing
    assert cache.read_text().strip()
    again = make_ising(lats, max_record=8)
    assert again.autotune(sweeps_per_trial=2) == choice


def test_checkpoint_resume_bit_identical():
    lats = wl.uneven512(n=12, seed=5, emin=4, emax=8)
    a = make_ising(lats)
    a.sweep(5)
    blob = a.checkpoint()
    a.sweep(6, record=True)
    b = make_ising(lats, seed=SEED)
    b.restore(blob)
    assert b.t == 5
    b.sweep(6, record=True)
    assert torch.equal(a.spins, b.spins)
    assert np.array_equal(a.observables_host()[0], b.observables_host()[0])


def test_ising_extremes_beta_zero_and_large():
    lats = [dict(L=32, beta=0.0, J=1.0, h=0.0), dict(L=32, beta=50.0, J=1.0, h=0.0)]
    sim = make_ising(lats)
    init = [lattice_np(sim, i) for i in range(2)]
    sim.sweep(1)
    # beta = 0: every proposal accepted -> every spin flipped once
    assert np.array_equal(lattice_np(sim, 0), -init[0])
    ref = init[1].copy()
    oracle.ising_sweep(ref, 50.0, 1.0, 0.0, SEED, 1, 0)
    assert np.array_equal(lattice_np(sim, 1), ref)


def test_stats_bookkeeping_matches_recount_large():
    """Recorded statistics (accumulated from accepted flips) equal a recount
    of the final state -- a property that holds at any size."""
    lats = wl.uneven512(n=64, seed=9)
    sim = make_ising(lats)
    sim.sweep(5, record=True)
    st, _, _ = sim.observables(4, 1)
    assert torch.equal(st[0], sim.current_stats())


# --------------------------------------------------------------------- Potts
POTTS = [dict(L=L, q=q, beta=b, J=J) for L, q, b, J in [
    (16, 2, 0.8, 1.0), (32, 3, 1.0, 1.0), (64, 8, 1.2, 1.0), (10, 3, 1.0, 1.0), (48, 5, 0.9, -1.0),
    (128, 3, 1.005, 1.0), (256, 8, 1.2, 1.0), (32, 20, 2.0, 1.0), (8, 255, 1.0, 1.0)]]


@pytest.mark.parametrize("mode,graph", [(0, True), (0, False), (1, True)])
def test_potts_mixed_batch(mode, graph):
    sim = sm.Sim(sm.SPIN_POTTS, POTTS, seed=SEED, max_record=32)
    sim.set_launch(mode, graph, 0, 256)
    init = {}
    for i, d in enumerate(POTTS):
        init[i] = lattice_np(sim, i)
        assert np.array_equal(init[i], oracle.init_potts(d["L"], d["q"], SEED, i))
    sim.sweep(1, record=True)
    for i, d in enumerate(POTTS):
        oracle.potts_sweep(init[i], d["q"], d["beta"], d["J"], SEED, i, 0)
        assert np.array_equal(lattice_np(sim, i), init[i]), i
    sim.sweep(6, record=True)
    st, E, M = sim.observables_host(0, 7)
    qmax = max(d["q"] for d in POTTS)
    for i, d in enumerate(POTTS):
        ref = oracle.potts_run(init[i], d["q"], d["beta"], d["J"], SEED, i, 1, 6)
        assert np.array_equal(lattice_np(sim, i), init[i]), i
        assert np.array_equal(st[1:, i, :d["q"] + 1], ref), i
        assert not st[1:, i, d["q"] + 1:qmax + 1].any()
        N = d["L"] ** 2
        Mq = (d["q"] * ref[:, 1:].max(axis=1) - N) / ((d["q"] - 1) * N)
        np.testing.assert_allclose(M[1:, i], Mq.astype(np.float32), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(E[1:, i], (-d["J"] * ref[:, 0] / N).astype(np.float32), rtol=1e-6, atol=1e-7)


# ----------------------------------------------------------------------- CPM
def cpm_sim(p, seed=SEED, max_record=32):
    cpm = dict(J=p["J"], **{"lambda": p["lam"]}, target=p["target"], n_cells=p["n_cells"], T=p["T"],
               side=p["side"], cols=p["cols"])
    return sm.Sim(sm.SPIN_CPM, [dict(L=p["L"])], seed=seed, max_record=max_record, cpm=cpm)


def oracle_cpm(p):
    return oracle.CPM(L=p["L"], J=p["J"], lam=p["lam"], target=p["target"], n_cells=p["n_cells"],
                      T=p["T"], side=p["side"], cols=p["cols"])


@pytest.mark.parametrize("mode,graph", [(0, True), (0, False), (2, True)])
def test_cpm_paper_setup_matches_oracle(mode, graph):
    p = wl.cpm_paper()
    sim = cpm_sim(p)
    sim.set_launch(mode, graph)
    op = oracle_cpm(p)
    ids, types, vol = op.init(SEED, 0)
    ids = ids.copy()
    assert np.array_equal(lattice_np(sim, 0), ids)
    sim.sweep(5, record=True)
    ref = op.run(ids, vol, types, SEED, 0, 0, 5)
    assert np.array_equal(lattice_np(sim, 0), ids)
    st, E, M = sim.observables_host(0, 5)
    assert np.array_equal(st[:, 0, :], ref)


def test_cpm_full_size_two_steps_and_gradient():
    p = wl.cpm1024()
    sim = cpm_sim(p)
    op = oracle_cpm(p)
    ids, types, vol = op.init(SEED, 0)
    ids = ids.copy()
    sim.sweep(2, record=True)
    ref = op.run(ids, vol, types, SEED, 0, 0, 2)
    assert np.array_equal(lattice_np(sim, 0), ids)
    st = sim.observables_host(0, 2)[0]
    assert np.array_equal(st[:, 0, :], ref)


def test_cpm_launch_forms_hand_over_the_chain():
    """Persistent (one cooperative launch per call, grid barriers between the
    sub-steps) and per-sub-step launches alternate within one chain: the
    areas, their pending changes, the contact counters and the records carry
    over, so the chain is the oracle's throughout."""
    p = wl.cpm1024()
    sim = cpm_sim(p)
    op = oracle_cpm(p)
    ids, types, vol = op.init(SEED, 0)
    ids = ids.copy()
    for mode, n in [(2, 2), (0, 1), (2, 3), (0, 2)]:
        sim.set_launch(mode, True)
        sim.sweep(n, record=True)
    ref = op.run(ids, vol, types, SEED, 0, 0, 8)
    assert np.array_equal(lattice_np(sim, 0), ids)
    st = sim.observables_host(0, 8)[0]
    assert np.array_equal(st[:, 0, :], ref)
    assert np.array_equal(sim.current_stats().cpu().numpy()[0], ref[-1])


# --------------------------------------------------------------- gradients
def test_ising_grad_matches_oracle_estimator():
    from oracle import estimator
    lats = wl.fit256(n=4, L=32, beta=0.45, J=1.0, h=0.05)
    sim = make_ising(lats, max_record=400)
    sim.sweep(300, record=True)
    st = sim.observables_host(0, 300)[0]          # [T, n_lat, 2]
    b32 = float(np.float32(0.45))                 # the library takes beta as float
    for obs, name in [(0, "E"), (1, "M")]:
        g = sim.grad(100, 200, observable=obs).cpu().numpy()
        gp = sim.grad(100, 200, observable=obs, pool=True).cpu().numpy()
        for i in range(4):
            ref = estimator.ising_grad(st[100:, i][None], b32, 1.0, float(np.float32(0.05)), 32 * 32)
            np.testing.assert_allclose(g[i], [ref[(name, "J")], ref[(name, "h")]], rtol=1e-9, atol=1e-12)
        refp = estimator.ising_grad(np.transpose(st[100:], (1, 0, 2)), b32, 1.0, float(np.float32(0.05)), 1024)
        np.testing.assert_allclose(gp[0], [refp[(name, "J")], refp[(name, "h")]], rtol=1e-9, atol=1e-12)
    mom = sim.moments(100, 200).cpu().numpy()
    for i in range(4):
        X = st[100:, i].astype(np.int64)
        want = [len(X), X[:, 0].sum(), X[:, 1].sum(), (X[:, 0] ** 2).sum(), (X[:, 0] * X[:, 1]).sum(),
                (X[:, 1] ** 2).sum()]
        assert list(mom[i]) == want


def test_cpm_grad_matches_oracle_estimator():
    from oracle import estimator
    p = wl.cpm_paper()
    sim = cpm_sim(p, max_record=200)
    sim.sweep(150, record=True)
    st = sim.observables_host(0, 150)[0]
    g = sim.grad(50, 100).cpu().numpy()[0]
    ref = estimator.cpm_grad(st[50:, 0][None], p["J"], p["lam"], p["T"], p["L"] ** 2)
    pairs = estimator.cpm_pairs(3)
    want = [ref[("J", a, b)] for a, b in pairs] + [ref["lambda"], ref["A"]]
    np.testing.assert_allclose(g, want, rtol=1e-9, atol=1e-12)
    assert g[0] == 0.0  # J_00: medium-medium contacts never exist


# --------------------------------------------- full-size configurations
def test_uneven512_full_size_sampled():
    """The batched launch form of the benchmark, at full size; the oracle
    checks every lattice up to 256^2 and one lattice of each larger size."""
    lats = wl.uneven512()
    sim = make_ising(lats, max_record=8)
    init_sample = {}
    sizes_seen = {}
    for i, d in enumerate(lats):
        if d["L"] <= 256 or d["L"] not in sizes_seen:
            sizes_seen.setdefault(d["L"], i)
            init_sample[i] = lattice_np(sim, i)
    sim.sweep(2, record=True)
    st = sim.observables_host(0, 2)[0]
    for i, s0 in init_sample.items():
        d = lats[i]
        ref = oracle.ising_run(s0, d["beta"], d["J"], d["h"], SEED, i, 0, 2)
        assert np.array_equal(lattice_np(sim, i), s0), i
        assert np.array_equal(st[:, i, :], ref), i
    assert torch.equal(sim.observables(1, 1)[0][0], sim.current_stats())


# Potts lattices on the strip kernel (q <= 8, L in {512, 1024, 2048}) next to
# ones on the tile kernel (smaller L, or q > 8) in the same launch.
POTTS_STRIP = [dict(L=L, q=q, beta=b, J=J) for L, q, b, J in [
    (512, 2, 0.9, 1.0), (512, 3, 1.005, 1.0), (1024, 4, 1.1, 1.0), (512, 5, 1.2, -1.0),
    (512, 8, 1.3, 1.0), (2048, 3, 0.8, 1.0), (512, 12, 1.5, 1.0), (64, 3, 1.0, 1.0),
    (1024, 7, 0.0, 1.0), (512, 6, 4.0, 1.0)]]


@pytest.mark.parametrize("mode,tile,threads,graph", [(0, 0, 256, True), (0, 24, 512, False), (0, 8, 256, False),
                                                     (0, 64, 512, True), (0, 1, 256, False), (3, 0, 256, True)])
def test_potts_strip_batch(mode, tile, threads, graph):
    sim = sm.Sim(sm.SPIN_POTTS, POTTS_STRIP, seed=SEED, max_record=8)
    sim.set_launch(mode, graph, tile, threads)
    ref = {i: lattice_np(sim, i) for i in range(len(POTTS_STRIP))}
    sim.sweep(1, record=True)
    for i, d in enumerate(POTTS_STRIP):
        oracle.potts_sweep(ref[i], d["q"], d["beta"], d["J"], SEED, i, 0)
        assert np.array_equal(lattice_np(sim, i), ref[i]), (i, d)
    sim.sweep(3, record=True)
    st = sim.observables_host(0, 4)[0]
    qmax = max(d["q"] for d in POTTS_STRIP)
    for i, d in enumerate(POTTS_STRIP):
        first = oracle.potts_stats(ref[i], d["q"])
        rest = oracle.potts_run(ref[i], d["q"], d["beta"], d["J"], SEED, i, 1, 3)
        assert np.array_equal(lattice_np(sim, i), ref[i]), (i, d)
        assert np.array_equal(st[0, i, :d["q"] + 1], first), i
        assert np.array_equal(st[1:, i, :d["q"] + 1], rest), i
        assert not st[:, i, d["q"] + 1:qmax + 1].any()
    # sweeps without records keep the running statistics exact as well
    sim.sweep(3)
    cur = sim.current_stats().cpu().numpy()
    for i, d in enumerate(POTTS_STRIP):
        assert np.array_equal(cur[i, :d["q"] + 1], oracle.potts_stats(lattice_np(sim, i), d["q"])), i


@pytest.mark.parametrize("mode,graph", [(0, True), (0, False), (3, True)])
def test_potts_split_rows_between_the_sweeps_of_a_call(mode, graph):
    """Potts strip lattices, like Ising ones, stay in the split row form between
    the sweeps of one call: calls of 2, 4 and 5 sweeps continue the oracle's
    chain, with the recorded statistics of every sweep."""
    sim = sm.Sim(sm.SPIN_POTTS, POTTS_STRIP, seed=SEED, max_record=16)
    sim.set_launch(mode, graph, 0, 256)
    ref = {i: lattice_np(sim, i) for i in range(len(POTTS_STRIP))}
    t = 0
    for n in (2, 4, 5):
        sim.sweep(n, record=True)
        st = sim.observables_host(t, n)[0]
        for i, d in enumerate(POTTS_STRIP):
            exp = oracle.potts_run(ref[i], d["q"], d["beta"], d["J"], SEED, i, t, n)
            assert np.array_equal(lattice_np(sim, i), ref[i]), (n, i)
            assert np.array_equal(st[:, i, :d["q"] + 1], exp), (n, i)
        t += n


@pytest.mark.parametrize("q", [3, 8])
def test_potts_full_size_sampled(q):
    lats = wl.potts_batch(q)
    sim = sm.Sim(sm.SPIN_POTTS, lats, seed=SEED, max_record=4)
    pick = [0, 31, 63]
    init = {i: lattice_np(sim, i) for i in pick}
    sim.sweep(2, record=True)
    st = sim.observables_host(0, 2)[0]
    for i in pick:
        d = lats[i]
        ref = oracle.potts_run(init[i], q, d["beta"], d["J"], SEED, i, 0, 2)
        assert np.array_equal(lattice_np(sim, i), init[i])
        assert np.array_equal(st[:, i, :], ref)


def test_out_of_range_states_are_harmless():
    """Caller-supplied states outside the model's range (init_mode 1) must not
    make a kernel index outside its buffers; the run completes."""
    lats = [dict(L=32, q=3, beta=1.0, J=1.0), dict(L=10, q=3, beta=1.0, J=1.0)]
    spins = torch.randint(0, 256, (2048,), dtype=torch.uint8, device="cuda")
    sim = sm.Sim(sm.SPIN_POTTS, lats, seed=SEED, spins=spins, offsets=[0, 1024], init_mode=1, max_record=4)
    sim.sweep(3, record=True)
    torch.cuda.synchronize()
    p = wl.cpm_paper()
    ids = torch.randint(-50, 5000, (p["L"] * p["L"],), dtype=torch.int32, device="cuda")
    cpm = dict(J=p["J"], **{"lambda": p["lam"]}, target=p["target"], n_cells=p["n_cells"], T=p["T"],
               side=p["side"], cols=p["cols"])
    cs = sm.Sim(sm.SPIN_CPM, [dict(L=p["L"])], seed=SEED, spins=ids, init_mode=1, max_record=4, cpm=cpm)
    cs.sweep(2, record=True)
    torch.cuda.synchronize()


# ------------------------------------------------------------ triangular lattice
TRI = [dict(L=L, beta=b, J=J, h=h, geometry=1) for L, b, J, h in [
    (6, 0.3, 1.0, 0.0), (12, 0.27, 1.0, 0.05), (48, 0.35, -1.0, 0.1), (96, 0.27, 1.0, 0.0)]]


@pytest.mark.parametrize("mode,graph", [(0, True), (0, False), (1, False)])
def test_triangular_lattices_next_to_square_ones(mode, graph):
    lats = TRI + [dict(L=64, beta=0.44, J=1.0, h=0.0), dict(L=10, beta=0.3, J=1.0, h=0.02)]
    sim = make_ising(lats, max_record=16)
    sim.set_launch(mode, graph, 0, 256)
    init = {i: lattice_np(sim, i) for i in range(len(lats))}
    st0 = sim.current_stats().cpu().numpy()
    for i, d in enumerate(lats):
        ref = oracle.tri_stats(init[i]) if d.get("geometry") else oracle.ising_stats(init[i])
        assert np.array_equal(st0[i], ref), i
    sim.sweep(1, record=True)
    sim.sweep(4, record=True)
    st = sim.observables_host(0, 5)[0]
    for i, d in enumerate(lats):
        s = init[i].copy()
        run = oracle.tri_run if d.get("geometry") else oracle.ising_run
        ref = run(s, d["beta"], d["J"], d["h"], SEED, i, 0, 5)
        assert np.array_equal(lattice_np(sim, i), s), (i, d)
        assert np.array_equal(st[:, i, :], ref), (i, d)


def test_load_recomputes_the_running_statistics():
    """spin_load_spins recounts the statistics of the loaded state: storing and
    loading back reproduces the sweeps' bookkeeping exactly (this pins the
    byte-parallel recount of the vectorisable lattices), and after loading an
    unrelated state the records follow the oracle chain from that state."""
    lats = wl.uneven512(n=48, seed=4) + [dict(L=10, beta=0.3, J=1.0, h=0.05),
                                         dict(L=48, beta=0.3, J=1.0, h=0.0, geometry=1)]
    sim = make_ising(lats, max_record=8)
    sim.sweep(5, record=True)
    torch.cuda.synchronize()
    kept = sim.current_stats().clone()
    span = int(sim.spins.numel())
    host = torch.zeros(span, dtype=torch.int8).pin_memory()
    sim.store_spins(host)
    sim.load_spins(host)
    torch.cuda.synchronize()
    assert torch.equal(sim.current_stats(), kept)
    rng = np.random.default_rng(3)
    new = torch.from_numpy(rng.choice(np.array([-1, 1], dtype=np.int8), size=span)).pin_memory()
    sim.load_spins(new)
    torch.cuda.synchronize()
    cur = sim.current_stats().cpu().numpy()
    pick = [0, 17, 47, len(lats) - 2, len(lats) - 1]
    init = {i: lattice_np(sim, i) for i in pick}
    for i in pick:
        stats = oracle.tri_stats if lats[i].get("geometry") else oracle.ising_stats
        assert np.array_equal(cur[i], stats(init[i])), i
    first = sim.n_records
    sim.sweep(2, record=True)
    st = sim.observables_host(first, 2)[0]
    for i in pick:
        d = lats[i]
        run = oracle.tri_run if d.get("geometry") else oracle.ising_run
        ref = run(init[i], d["beta"], d["J"], d["h"], SEED, i, 5, 2)
        assert np.array_equal(st[:, i, :], ref), i


@pytest.mark.parametrize("graph", [True, False])
def test_triangular_resident_form(graph):
    """Batches of triangular lattices only may run resident in shared memory
    (launch mode 2): the same chain, records every sweep."""
    lats = TRI + [dict(L=192, beta=0.3, J=1.0, h=-0.02, geometry=1)]
    sim = make_ising(lats, max_record=16)
    sim.set_launch(2, graph, 0, 512)
    init = {i: lattice_np(sim, i) for i in range(len(lats))}
    sim.sweep(3, record=True)
    sim.sweep(2, record=True)
    st = sim.observables_host(0, 5)[0]
    for i, d in enumerate(lats):
        s = init[i].copy()
        ref = oracle.tri_run(s, d["beta"], d["J"], d["h"], SEED, i, 0, 5)
        assert np.array_equal(lattice_np(sim, i), s), i
        assert np.array_equal(st[:, i, :], ref), i
    assert np.array_equal(sim.current_stats().cpu().numpy()[:, :], st[-1])


def test_resident_form_with_1024_threads():
    """The square-lattice resident kernel also runs 1024-thread blocks (one
    lattice per SM with twice the warps); the chain is the oracle's."""
    lats = wl.fit256(n=6, L=64, beta=0.44, J=1.0, h=0.02) + [dict(L=256, beta=0.3, J=1.0, h=0.0)]
    sim = make_ising(lats, max_record=8)
    sim.set_launch(2, True, 0, 1024)
    assert sim.get_launch()["threads"] == 1024
    init = {i: lattice_np(sim, i) for i in range(len(lats))}
    sim.sweep(3, record=True)
    out, stats = oracle_ising_chain(lats, SEED, init, 0, 3)
    st = sim.observables_host(0, 3)[0]
    for i in range(len(lats)):
        assert np.array_equal(lattice_np(sim, i), out[i]), i
        assert np.array_equal(st[:, i, :], stats[i]), i
    sim.set_launch(0, True, 0, 0)       # back to the batched form: threads fall back to 512
    assert sim.get_launch()["threads"] == 512


@pytest.mark.parametrize("mode", [0, 1])
def test_large_lattices_against_the_oracle(mode):
    """Lattices far above the strip sizes (4096^2 and 8192^2 Ising, 4096^2 Potts
    with q = 5): work items with recomputed halos in the batched form and
    per-lattice launches in the plain form, two sweeps against the oracle."""
    lats = [dict(L=4096, beta=0.44, J=1.0, h=0.01), dict(L=8192, beta=0.3, J=1.0, h=0.0)]
    sim = make_ising(lats, max_record=4)
    sim.set_launch(mode, True, 0, 256)
    init = {i: lattice_np(sim, i) for i in range(len(lats))}
    sim.sweep(2, record=True)
    out, stats = oracle_ising_chain(lats, SEED, init, 0, 2)
    st = sim.observables_host(0, 2)[0]
    for i in range(len(lats)):
        assert np.array_equal(lattice_np(sim, i), out[i]), i
        assert np.array_equal(st[:, i, :], stats[i]), i
    del sim
    pl = [dict(L=4096, q=5, beta=1.1, J=1.0)]
    ps = sm.Sim(sm.SPIN_POTTS, pl, seed=SEED, max_record=4)
    ps.set_launch(mode, True, 0, 256)
    p0 = ps.lattice(0).cpu().numpy().copy()
    ps.sweep(2, record=True)
    ref = oracle.potts_run(p0, 5, 1.1, 1.0, SEED, 0, 0, 2)
    assert np.array_equal(ps.lattice(0).cpu().numpy(), p0)
    assert np.array_equal(ps.observables_host(0, 2)[0][:, 0, :], ref)


def test_empty_calls_change_nothing():
    """Zero sweeps, zero records and zero-length reads are valid no-ops; a
    gradient needs two records."""
    lats = [dict(L=16, beta=0.4, J=1.0, h=0.0), dict(L=512, beta=0.3, J=1.0, h=0.1)]
    sim = make_ising(lats, max_record=4)
    before = [lattice_np(sim, i) for i in range(2)]
    st0 = sim.current_stats().clone()
    sim.sweep(0, record=True)
    assert sim.t == 0 and sim.n_records == 0
    assert all(np.array_equal(lattice_np(sim, i), before[i]) for i in range(2))
    assert torch.equal(sim.current_stats(), st0)
    st, E, M = sim.observables_host(0, 0)
    assert st.shape == (0, 2, 2) and E.size == 0 and M.size == 0
    sim.sweep(1, record=True)
    with pytest.raises(sm.SpinError):
        sim.grad(0, 1)
    mom = sim.moments(0, 1).cpu().numpy()
    assert list(mom[:, 0]) == [1, 1]            # one sample per lattice


def test_bit_packed_load_of_large_lattices():
    """The unpack kernel's row walk over several grid strides: lattices of 2048
    and 1056 (33 words per row, so a stride is not a whole number of rows) and
    96; the loaded spins are the bits and the recounted statistics the
    oracle's."""
    lats = [dict(L=L, beta=0.44, J=1.0, h=0.0) for L in (2048, 1056, 96)]
    sim = make_ising(lats, max_record=4)
    nw = sim.packed_words
    span = int(sim.spins.numel())
    rng = np.random.default_rng(9)
    new = torch.from_numpy(rng.integers(-2 ** 31, 2 ** 31, nw, dtype=np.int64).astype(np.int32)).pin_memory()
    sim.load_spins_packed(new)
    torch.cuda.synchronize()
    nb = np.unpackbits(new.numpy().view(np.uint8), bitorder="little")[:span]
    cur = sim.current_stats().cpu().numpy()
    for i, (off, d) in enumerate(zip(sim.offsets, lats)):
        L = d["L"]
        want = np.where(nb[off:off + L * L] == 1, -1, 1).astype(np.int8).reshape(L, L)
        got = lattice_np(sim, i)
        assert np.array_equal(got, want), L
        assert list(cur[i]) == list(oracle.ising_stats(want)), L


def test_bit_packed_transfer():
    """One bit per spin on the host: a store packs exactly the lattices'
    signs (bits outside them 0), a load unpacks into the lattices only (other
    bytes of the span untouched), recounts the statistics, and the chain from the
    loaded state is the oracle's."""
    lats = MIXED[:8]
    sim = make_ising(lats, max_record=8)
    sim.sweep(3, record=True)
    nw = sim.packed_words
    span = int(sim.spins.numel())
    assert nw == (span + 31) // 32
    words = torch.zeros(nw, dtype=torch.int32).pin_memory()
    sim.store_spins_packed(words)
    torch.cuda.synchronize()
    full = sim.spins.cpu().numpy()
    inside = np.zeros(nw * 32, dtype=bool)
    for off, d in zip(sim.offsets, lats):
        inside[off:off + d["L"] ** 2] = True
    bits = np.zeros(nw * 32, dtype=np.uint8)
    bits[:span] = (full < 0) & inside[:span]
    assert np.array_equal(words.numpy().view(np.uint8), np.packbits(bits, bitorder="little"))
    rng = np.random.default_rng(8)
    new = torch.from_numpy(rng.integers(-2 ** 31, 2 ** 31, nw, dtype=np.int64).astype(np.int32)).pin_memory()
    before = sim.spins.cpu().numpy()
    sim.load_spins_packed(new)
    torch.cuda.synchronize()
    after = sim.spins.cpu().numpy()
    nb = np.unpackbits(new.numpy().view(np.uint8), bitorder="little")[:span]
    want = np.where(nb == 1, -1, 1).astype(np.int8)
    assert np.array_equal(after[inside[:span]], want[inside[:span]])
    assert np.array_equal(after[~inside[:span]], before[~inside[:span]])
    init = {i: lattice_np(sim, i) for i in range(len(lats))}
    cur = sim.current_stats().cpu().numpy()
    for i in range(len(lats)):
        assert list(cur[i]) == list(oracle.ising_stats(init[i])), i
    first = sim.n_records
    sim.sweep(2, record=True)
    out, stats = oracle_ising_chain(lats, SEED, init, 3, 2)
    st = sim.observables_host(first, 2)[0]
    for i in range(len(lats)):
        assert np.array_equal(lattice_np(sim, i), out[i]), i
        assert np.array_equal(st[:, i, :], stats[i]), i


@pytest.mark.parametrize("mode,graph,n", [(0, True, 1), (0, True, 2), (0, True, 3), (0, False, 3), (3, True, 1),
                                          (2, True, 1)])
def test_sweep_packed_equals_load_sweep_store(mode, graph, n):
    """spin_sweep_packed (upload, n sweeps, download in one call; an odd n in a
    ping-pong form starts from the other buffer and needs no final copy) gives
    the bits, spins, records and counter of load + sweep + store, and the
    oracle's chain from the loaded state."""
    lats = ([dict(L=L, beta=b, J=1.0, h=h) for L, b, h in [(16, 0.3, 0.0), (64, 0.44, 0.05), (128, 0.5, 0.0),
                                                            (256, 0.4, -0.02)]] if mode == 2 else
            [dict(L=L, beta=b, J=1.0, h=h) for L, b, h in [(512, 0.44, 0.0), (16, 0.3, 0.1), (1024, 0.5, -0.02),
                                                            (10, 0.4, 0.0), (64, 0.6, 0.0), (2048, 0.35, 0.01)]])
    a, b = make_ising(lats, max_record=8), make_ising(lats, max_record=8)
    for x in (a, b):
        x.set_launch(mode, graph, -1, 512)
        x.sweep(2, record=True)
    nw = a.packed_words
    rng = np.random.default_rng(31 + n)
    bits = torch.from_numpy(rng.integers(-2 ** 31, 2 ** 31, nw, dtype=np.int64).astype(np.int32)).pin_memory()
    out_a = torch.zeros(nw, dtype=torch.int32).pin_memory()
    out_b = torch.ones(nw, dtype=torch.int32).pin_memory()
    a.load_spins_packed(bits)
    loaded = {i: lattice_np(a, i) for i in range(len(lats))}
    a.sweep(n, record=True)
    a.store_spins_packed(out_a)
    b.sweep_packed(bits, out_b, n, record=True)
    torch.cuda.synchronize()
    assert torch.equal(out_a, out_b)
    assert torch.equal(a.spins, b.spins)
    assert a.t == b.t == 2 + n and a.n_records == b.n_records == 2 + n
    assert np.array_equal(a.observables_host(2, n)[0], b.observables_host(2, n)[0])
    assert torch.equal(a.current_stats(), b.current_stats())
    st = b.observables_host(2, n)[0]
    for i in (0, 1, len(lats) - 1):
        d, s = lats[i], loaded[i].copy()
        ref = oracle.ising_run(s, d["beta"], d["J"], d["h"], SEED, i, 2, n)
        assert np.array_equal(lattice_np(b, i), s), i
        assert np.array_equal(st[:, i], ref), i


def test_sweep_packed_without_buffers_is_a_sweep():
    lats = MIXED[:6]
    a, b = make_ising(lats, max_record=4), make_ising(lats, max_record=4)
    a.sweep(3, record=True)
    b.sweep_packed(None, None, 3, record=True)
    torch.cuda.synchronize()
    assert torch.equal(a.spins, b.spins)
    assert np.array_equal(a.observables_host(0, 3)[0], b.observables_host(0, 3)[0])


def test_sweep_packed_full_size_uneven512():
    """The one-sweep bit-layout path on the benchmark's batch (512 lattices,
    the strip kernel reading and writing packed rows) against load + sweep +
    store, twice in a row."""
    lats = wl.uneven512()
    a, b = make_ising(lats, max_record=4), make_ising(lats, max_record=4)
    for x in (a, b):
        x.set_launch(0, True, 0, 512)
    nw = a.packed_words
    rng = np.random.default_rng(77)
    bits = torch.from_numpy(rng.integers(-2 ** 31, 2 ** 31, nw, dtype=np.int64).astype(np.int32)).pin_memory()
    for k in range(2):
        out_a = torch.zeros(nw, dtype=torch.int32).pin_memory()
        out_b = torch.ones(nw, dtype=torch.int32).pin_memory()
        a.load_spins_packed(bits)
        a.sweep(1, record=True)
        a.store_spins_packed(out_a)
        b.sweep_packed(bits, out_b, 1, record=True)
        torch.cuda.synchronize()
        assert torch.equal(out_a, out_b), k
        assert torch.equal(a.spins, b.spins), k
        assert np.array_equal(a.observables_host(k, 1)[0], b.observables_host(k, 1)[0]), k
        bits = out_b.clone().pin_memory()


def test_sweep_packed_offsets_off_the_bit_layout_and_edge_calls():
    """A strip lattice whose packed rows would not start on 16-byte boundaries
    (offset % 128 != 0) takes the unpack / pack path; a call with no sweep is a
    load and a store; one with only an output is a sweep and a store."""
    lats = [dict(L=16, beta=0.3, J=1.0, h=0.0), dict(L=6, beta=0.5, J=1.0, h=0.1),
            dict(L=512, beta=0.44, J=1.0, h=0.0), dict(L=1024, beta=0.5, J=1.0, h=-0.02)]
    offsets, _ = sm.pack_offsets([d["L"] for d in lats], 1, 32)
    assert offsets[2] % 128 != 0
    a, b = make_ising(lats, max_record=8, offsets=offsets), make_ising(lats, max_record=8, offsets=offsets)
    nw = a.packed_words
    rng = np.random.default_rng(5)
    bits = torch.from_numpy(rng.integers(-2 ** 31, 2 ** 31, nw, dtype=np.int64).astype(np.int32)).pin_memory()
    out_a, out_b = (torch.zeros(nw, dtype=torch.int32).pin_memory() for _ in range(2))
    a.load_spins_packed(bits)
    a.sweep(1, record=True)
    a.store_spins_packed(out_a)
    b.sweep_packed(bits, out_b, 1, record=True)
    torch.cuda.synchronize()
    assert torch.equal(out_a, out_b) and torch.equal(a.spins, b.spins)
    assert np.array_equal(a.observables_host(0, 1)[0], b.observables_host(0, 1)[0])
    # no sweep: load then store
    out_c = torch.ones(nw, dtype=torch.int32).pin_memory()
    b.sweep_packed(bits, out_c, 0)
    a.load_spins_packed(bits)
    a.store_spins_packed(out_a)
    torch.cuda.synchronize()
    assert torch.equal(out_a, out_c) and torch.equal(a.spins, b.spins)
    assert torch.equal(a.current_stats(), b.current_stats())
    # only an output: sweeps then a store
    a.sweep(2, record=True)
    a.store_spins_packed(out_a)
    b.sweep_packed(None, out_c, 2, record=True)
    torch.cuda.synchronize()
    assert torch.equal(out_a, out_c) and torch.equal(a.spins, b.spins)
    assert a.t == b.t == 3

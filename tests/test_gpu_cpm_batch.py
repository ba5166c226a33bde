"""Batched cellular Potts (many lattices of the paper's cell-sorting size in
one launch) against the CPU oracle, lattice by lattice, bit for bit: the
initial state, the ids, areas and per-step statistics after every call, a
batch larger than one wave of blocks (sampled), caller-given cell types, and
lattice 0 against the single-lattice context (same Philox stream)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2304_01772_gb300 as sm
from paper_2304_01772_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SEED = 0xBA7C4C0FFEE


def paper_cpm(**over):
    p = wl.cpm_paper()
    p.update(over)
    return p


def as_cpm(p):
    return dict(J=p["J"], **{"lambda": p["lam"]}, target=p["target"], n_cells=p["n_cells"], T=p["T"],
                side=p["side"], cols=p["cols"], **({"cell_type": p["cell_type"]} if "cell_type" in p else {}))


def oracle_model(p):
    return oracle.CPM(L=p["L"], J=p["J"], lam=p["lam"], target=p["target"], n_cells=p["n_cells"], T=p["T"],
                      side=p["side"], cols=p["cols"])


@pytest.mark.parametrize("over", [{}, dict(T=3.0, lam=2), dict(L=32, n_cells=16, side=6, cols=4, target=36)])
def test_batch_init_and_steps_match_oracle(over):
    p = paper_cpm(**over)
    B = 5
    batch = sm.CPMBatch(B, p["L"], as_cpm(p), seed=SEED)
    op = oracle_model(p)
    ref = [list(op.init(SEED, b)) for b in range(B)]
    for b in range(B):
        ids, types, vol = ref[b]
        assert np.array_equal(batch.ids[b].cpu().numpy().ravel(), np.ravel(ids)), b
        assert np.array_equal(batch.types[b].cpu().numpy(), types), b
        assert np.array_equal(batch.areas[b].cpu().numpy(), vol), b
    st1 = batch.run(2, record=True).cpu().numpy()
    st2 = batch.run(3, record=True).cpu().numpy()
    for b in range(B):
        ids, types, vol = ref[b]
        ids = ids.copy()
        r1 = op.run(ids, vol, types, SEED, b, 0, 2)
        r2 = op.run(ids, vol, types, SEED, b, 2, 3)
        assert np.array_equal(st1[:, b, :], r1), b
        assert np.array_equal(st2[:, b, :], r2), b
        assert np.array_equal(batch.ids[b].cpu().numpy().ravel(), np.ravel(ids)), b
        assert np.array_equal(batch.areas[b].cpu().numpy(), vol), b


def test_large_batch_sampled():
    """More lattices than blocks in flight: the grid-stride loop."""
    p = paper_cpm()
    B = 2000
    batch = sm.CPMBatch(B, p["L"], as_cpm(p), seed=SEED)
    batch.run(2)
    op = oracle_model(p)
    for b in (0, 1217, 1999):
        ids, types, vol = op.init(SEED, b)
        ids = ids.copy()
        op.run(ids, vol, types, SEED, b, 0, 2, record=False)
        assert np.array_equal(batch.ids[b].cpu().numpy().ravel(), np.ravel(ids)), b
        assert np.array_equal(batch.areas[b].cpu().numpy(), vol), b


def test_given_cell_types_apply_to_every_lattice():
    p = paper_cpm()
    types = np.array([0] + [1 + (c % 2) for c in range(1, p["n_cells"] + 1)], dtype=np.uint8)
    batch = sm.CPMBatch(3, p["L"], dict(as_cpm(p), cell_type=types), seed=SEED)
    for b in range(3):
        assert np.array_equal(batch.types[b].cpu().numpy(), types)
    batch.run(1)
    torch.cuda.synchronize()


def test_lattice_zero_equals_the_single_lattice_context():
    p = paper_cpm()
    batch = sm.CPMBatch(4, p["L"], as_cpm(p), seed=SEED)
    sim = sm.Sim(sm.SPIN_CPM, [dict(L=p["L"])], seed=SEED, max_record=4, cpm=as_cpm(p))
    st = batch.run(3, record=True)
    sim.sweep(3, record=True)
    assert torch.equal(batch.ids[0].reshape(-1), sim.lattice(0).reshape(-1))
    assert torch.equal(st[:, 0, :], sim.observables(0, 3)[0][:, 0, :])


def test_out_of_range_ids_and_types_are_harmless():
    p = paper_cpm()
    batch = sm.CPMBatch(2, p["L"], as_cpm(p), seed=SEED)
    batch.ids.copy_(torch.randint(-50, 5000, batch.ids.shape, dtype=torch.int32, device="cuda"))
    batch.types.copy_(torch.randint(0, 256, batch.types.shape, dtype=torch.uint8, device="cuda"))
    batch.run(2, record=True)
    torch.cuda.synchronize()

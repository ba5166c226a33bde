"""Failure detection on the GPU without a fault: the one device-side wait of
the library (the grid barrier of the CPM persistent form) is bounded.  A
cooperative self-test launch whose barriers wait for one block more than it
has cannot complete; every block must give up after the bounded wait (1 s),
the call must return SPIN_ETIMEOUT, and the device must stay usable."""
import time

import numpy as np
import pytest

import oracle
import paper_2304_01772_gb300 as sm
from paper_2304_01772_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SPIN_ETIMEOUT = -4
SEED = 0x5EED1234ABCD


def test_grid_barrier_completes_or_reports_a_timeout():
    assert sm.barrier_selftest(64, 0, 500) == 0
    t0 = time.perf_counter()
    assert sm.barrier_selftest(8, 1, 3) == SPIN_ETIMEOUT
    dt = time.perf_counter() - t0
    assert 0.9 < dt < 30, dt
    assert sm.barrier_selftest(16, 0, 100) == 0   # the barrier words start afresh


def test_device_usable_after_a_timed_out_barrier():
    assert sm.barrier_selftest(4, 2, 1) == SPIN_ETIMEOUT
    p = wl.cpm_paper()
    cpm = dict(J=p["J"], **{"lambda": p["lam"]}, target=p["target"], n_cells=p["n_cells"], T=p["T"],
               side=p["side"], cols=p["cols"])
    sim = sm.Sim(sm.SPIN_CPM, [dict(L=p["L"])], seed=SEED, max_record=8, cpm=cpm)
    sim.set_launch(2, True)
    op = oracle.CPM(L=p["L"], J=p["J"], lam=p["lam"], target=p["target"], n_cells=p["n_cells"], T=p["T"],
                    side=p["side"], cols=p["cols"])
    ids, types, vol = op.init(SEED, 0)
    ids = ids.copy()
    sim.sweep(3, record=True)
    ref = op.run(ids, vol, types, SEED, 0, 0, 3)
    assert np.array_equal(sim.lattice(0).cpu().numpy(), ids)
    assert np.array_equal(sim.observables_host(0, 3)[0][:, 0, :], ref)

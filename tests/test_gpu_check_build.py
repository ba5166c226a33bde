"""The bounds-checked build (libspinmc_check.so, -DSPIN_CHECK) on the GPU.

Its kernels check every work-list entry, shared-memory ring and queue index
and table address before use and record a code instead of trapping.  Run in
a child process that loads that build: small and strip-sized Ising lattices,
Potts lattices on the strip and tile kernels, a paper-size CPM lattice and
the allocation-free entry point must match the oracle bit for bit with no
check recorded."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle
import paper_2304_01772_gb300 as sm
from paper_2304_01772_gb300 import workloads as wl
assert sm.library_path().endswith("libspinmc_check.so")
built, code = sm.check_status()
assert built and code == 0, (built, code)
SEED = 99
lats = [dict(L=L, beta=b, J=1.0, h=h) for L, b, h in [(4, 0.3, 0.0), (8, 0.5, 0.1), (16, 0.44, 0.0),
        (10, 0.4, -0.1), (64, 0.44, 0.02), (512, 0.41, 0.0), (1024, 0.5, -0.01), (2048, 0.3, 0.0)]]
for mode, threads in ((0, 512), (0, 256), (3, 256), (1, 256)):
    sim = sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=4)
    sim.set_launch(mode, True, 0, threads)
    init = [sim.lattice(i).cpu().numpy().copy() for i in range(len(lats))]
    sim.sweep(3, record=True)
    st = sim.observables_host(0, 3)[0]
    for i, d in enumerate(lats):
        ref = oracle.ising_run(init[i], d["beta"], d["J"], d["h"], SEED, i, 0, 3)
        assert np.array_equal(sim.lattice(i).cpu().numpy(), init[i]), (mode, i)
        assert np.array_equal(st[:, i], ref), (mode, i)
    assert sm.check_status() == (True, 0), (mode, sm.check_status())
# one sweep between bit-packed transfers (strip kernel reading and writing packed rows)
pa, pb = (sm.Sim(sm.SPIN_ISING, lats, seed=SEED, max_record=4) for _ in range(2))
nwp = pa.packed_words
bits = torch.from_numpy(np.random.default_rng(5).integers(-2 ** 31, 2 ** 31, nwp, dtype=np.int64)
                        .astype(np.int32)).pin_memory()
oa, ob = torch.zeros(nwp, dtype=torch.int32).pin_memory(), torch.ones(nwp, dtype=torch.int32).pin_memory()
pa.load_spins_packed(bits)
pa.sweep(1, record=True)
pa.store_spins_packed(oa)
pb.sweep_packed(bits, ob, 1, record=True)
torch.cuda.synchronize()
assert torch.equal(oa, ob) and torch.equal(pa.spins, pb.spins)
assert sm.check_status() == (True, 0), ("packed", sm.check_status())
small = [dict(L=L, beta=0.4, J=1.0, h=0.0) for L in (16, 32, 64, 128)]
for cs in (1, 2, 4):   # one CTA per lattice, or a cluster of 2 or 4
    r = sm.Sim(sm.SPIN_ISING, small, seed=SEED, max_record=4)
    r.set_launch(2, False, cs, 256)
    init = [r.lattice(i).cpu().numpy().copy() for i in range(len(small))]
    r.sweep(3, record=True)
    for i, d in enumerate(small):
        oracle.ising_run(init[i], d["beta"], d["J"], d["h"], SEED, i, 0, 3)
        assert np.array_equal(r.lattice(i).cpu().numpy(), init[i]), (cs, i)
    assert sm.check_status() == (True, 0), (cs, sm.check_status())
potts = [dict(L=L, q=q, beta=1.0, J=1.0) for L, q in ((512, 3), (1024, 8), (64, 3), (48, 5))]
ps = sm.Sim(sm.SPIN_POTTS, potts, seed=SEED, max_record=4)
p0 = [ps.lattice(i).cpu().numpy().copy() for i in range(len(potts))]
ps.sweep(2, record=True)
for i, d in enumerate(potts):
    oracle.potts_run(p0[i], d["q"], d["beta"], d["J"], SEED, i, 0, 2, record=False)
    assert np.array_equal(ps.lattice(i).cpu().numpy(), p0[i]), i
p = wl.cpm_paper()
cs = sm.Sim(sm.SPIN_CPM, [dict(L=p["L"])], seed=SEED, cpm=dict(J=p["J"], **{"lambda": p["lam"]},
            target=p["target"], n_cells=p["n_cells"], T=p["T"], side=p["side"], cols=p["cols"]), max_record=4)
cs.sweep(3, record=True)
op = oracle.CPM(L=p["L"], J=p["J"], lam=p["lam"], target=p["target"], n_cells=p["n_cells"], T=p["T"],
                side=p["side"], cols=p["cols"])
ids, types, vol = op.init(SEED, 0)
ids = ids.copy()
op.run(ids, vol, types, SEED, 0, 0, 3, record=False)
assert np.array_equal(cs.lattice(0).cpu().numpy(), ids)
torch.cuda.synchronize()
assert sm.check_status() == (True, 0), sm.check_status()
print("check build: ok")
'''


def test_bounds_checked_build_matches_the_oracle_with_no_check_recorded():
    from paper_2304_01772_gb300 import build
    lib = build.build(variant="check")
    env = dict(os.environ, SPINMC_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "check build: ok" in r.stdout


def test_the_default_build_reports_no_checks():
    import paper_2304_01772_gb300 as sm
    if os.environ.get("SPINMC_LIBRARY"):
        pytest.skip("a test build is loaded")
    assert sm.check_status() == (False, 0)

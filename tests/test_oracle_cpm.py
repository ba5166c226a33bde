"""Pins for the oracle's cellular Potts chain (CPU only).

The CPM's stationary law is not a Boltzmann law of H (copy attempts are not
symmetric proposals, and area terms use snapshot areas), so the pins here are
exact bookkeeping identities and an independent brute-force replica."""
import math

import numpy as np
import pytest

import oracle
from tests import exact

J_PAPER = [[0, 16, 16], [16, 2, 11], [16, 11, 14]]   # medium, light, dark (paper's table)
MOORE = [(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]


def small_cpm(T=8.0, lam=1, target=16):
    return oracle.CPM(L=24, J=J_PAPER, lam=lam, target=target, n_cells=9, T=T, side=4, cols=3)


def _replica_cpm_substep(ids, vol, types, p, seed, lat, t, c):
    """One colour sub-step from the definitions: adhesion change from the full
    adhesion energy; area change from the snapshot areas at sub-step start."""
    L = ids.shape[0]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    snap = vol.copy()
    Jt = np.asarray(p.J)
    for y in range(L):
        for x in range(L):
            if (x & 1) | ((y & 1) << 1) != c:
                continue
            k = (y >> 1) * (L // 2) + (x >> 1)
            r = oracle.philox4x32_10([k >> 1, lat, t, c], key)
            u0, u1 = int(r[2 * (k & 1)]), int(r[2 * (k & 1) + 1])
            dx, dy = MOORE[u1 >> 29]
            sg = int(ids[y, x])
            sp = int(ids[(y + dy) % L, (x + dx) % L])
            if sp == sg:
                continue
            a0 = exact.cpm_adhesion(ids, types, Jt)
            ids[y, x] = sp
            a1 = exact.cpm_adhesion(ids, types, Jt)
            ids[y, x] = sg
            area = lambda cid, a: 0 if cid == 0 else p.lam * (a - p.target) ** 2
            dH = (a1 - a0) + area(sp, snap[sp] + 1) - area(sp, snap[sp]) \
                + area(sg, snap[sg] - 1) - area(sg, snap[sg])
            acc = dH <= 0 or u0 < max(math.floor(math.exp(-dH / float(np.float32(p.T))) * 2.0 ** 32), 1)
            if acc:
                ids[y, x] = sp
                vol[sp] += 1
                vol[sg] -= 1


def test_cpm_init_geometry_and_types():
    p = oracle.CPM(L=1024, J=J_PAPER, lam=1, target=400, n_cells=2000, T=10.0, side=20, cols=50)
    ids, types, vol = p.init(0)
    assert ids.max() == 2000 and vol[1:].min() == 400 and vol[1:].max() == 400
    assert vol[0] == 1024 * 1024 - 2000 * 400
    assert ids[112, 12] == 1 and ids[111, 12] == 0 and ids[112, 11] == 0
    assert ids[112 + 799, 12 + 999] == 2000 and ids[112 + 800, 12 + 999] == 0
    assert types[0] == 0 and set(np.unique(types[1:])) == {1, 2}
    assert 800 < int((types[1:] == 1).sum()) < 1200


def test_cpm_substeps_match_bruteforce_replica():
    p = small_cpm()
    ids, types, vol = p.init(77, 2)
    ids = ids.copy()
    rid, rvol = ids.copy(), vol.copy()
    for t in range(2):
        for c in range(4):
            p.substep(ids, vol, types, 77, 2, t, c)
            _replica_cpm_substep(rid, rvol, types, p, 77, 2, t, c)
            assert np.array_equal(ids, rid), (t, c)
            assert np.array_equal(vol, rvol)


def test_cpm_volume_is_histogram_after_every_substep():
    p = small_cpm()
    ids, types, vol = p.init(3)
    ids = ids.copy()
    for t in range(20):
        for c in range(4):
            p.substep(ids, vol, types, 3, 0, t, c)
            assert np.array_equal(vol, np.bincount(ids.ravel(), minlength=p.n_cells + 1))


def test_cpm_stats_definition():
    p = small_cpm()
    ids, types, vol = p.init(5)
    ids = ids.copy()
    p.run(ids, vol, types, 5, 0, 0, 10, record=False)
    st = p.stats(ids, vol, types)
    pairs = [(a, b) for a in range(3) for b in range(a, 3)]
    Jt = np.asarray(J_PAPER)
    adh = sum(Jt[a, b] * st[i] for i, (a, b) in enumerate(pairs))
    assert adh == exact.cpm_adhesion(ids, types, Jt)
    assert st[0] == 0  # medium is one cell: no medium-medium contacts
    d = vol[1:].astype(np.int64) - p.target
    assert st[len(pairs)] == int((d * d).sum()) and st[len(pairs) + 1] == int(d.sum())
    assert p.energy(ids, types) == adh + p.lam * int((d * d).sum())


def test_cpm_zero_temperature_never_goes_uphill():
    """At T -> 0 only dH <= 0 copies pass; with one accepted copy per cell per
    sub-step the snapshot area term is exact, so H never increases."""
    p = oracle.CPM(L=24, J=J_PAPER, lam=1, target=16, n_cells=9, T=1e-3, side=4, cols=3)
    ids, types, vol = p.init(9)
    ids = ids.copy()
    for t in range(10):
        for c in range(4):
            before = ids.copy()
            H0 = p.energy(ids, types)
            p.substep(ids, vol, types, 9, 0, t, c)
            changed = np.argwhere(before != ids)
            # every changed cell id changed at most once in this sub-step
            if len(changed):
                cells = np.concatenate([before[tuple(changed.T)], ids[tuple(changed.T)]])
                cells = cells[cells != 0]      # the medium has no area term
                if len(np.unique(cells)) == len(cells):
                    assert p.energy(ids, types) <= H0


def test_cpm_light_cells_leave_medium():
    """Cell sorting (Sec. "Cellular Potts model" results): light-medium contacts
    fall as light cells are engulfed by dark ones."""
    p = oracle.CPM(L=64, J=J_PAPER, lam=1, target=25, n_cells=36, T=8.0, side=5, cols=6)
    ids, types, vol = p.init(1)
    ids = ids.copy()
    st = p.run(ids, vol, types, 1, 0, 0, 400)
    lm = st[:, 1]  # pair (0, 1): medium-light
    assert lm[-50:].mean() < 0.7 * lm[:5].mean()

"""Pins of the triangular-lattice Ising oracle (other connectivities, Sec.
"Ising model"): a bit-exact replica whose energy change is a brute-force
difference of the Hamiltonian over an independently built six-neighbour bond
list, the (M, B) statistics recounted from that list, and exact enumeration
of the 3 x 3 periodic triangular lattice (2^9 states) against chain averages."""
import itertools
import math

import numpy as np

import oracle
from tests.exact import binned_stderr

SEED = 0x7121A9


def bonds(L):
    """Each nearest-neighbour pair of the triangular lattice once."""
    out = set()
    for y in range(L):
        for x in range(L):
            for dx, dy in [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)]:
                a, b = y * L + x, ((y + dy) % L) * L + (x + dx) % L
                out.add((min(a, b), max(a, b)))
    return sorted(out)


def energy(s, J, h, bl):
    f = s.ravel().astype(np.int64)
    return -J * sum(f[a] * f[b] for a, b in bl) - h * f.sum()


def test_replica_with_brute_force_energy_change():
    L, beta, J, h = 6, 0.4, 1.0, 0.1
    bl = bonds(L)
    assert len(bl) == 3 * L * L
    s0 = oracle.init_ising(L, SEED, 2)
    got = s0.copy()
    oracle.tri_sweep(got, beta, J, h, SEED, 2, 0)
    oracle.tri_sweep(got, beta, J, h, SEED, 2, 1)
    ref = s0.copy()
    key = [SEED & 0xFFFFFFFF, SEED >> 32]
    for t in range(2):
        for c in range(3):
            for y in range(L):
                for x in range(L):
                    if (x - y) % 3 != c:
                        continue
                    flipped = ref.copy()
                    flipped[y, x] = -flipped[y, x]
                    dE = float(energy(flipped, J, h, bl) - energy(ref, J, h, bl))
                    k = y * (L // 3) + x // 3
                    u = int(oracle.philox4x32_10([k >> 2, 2, t, c], key)[k & 3])
                    if dE <= 0 or u < oracle.accept_count(beta, dE):
                        ref = flipped
    np.testing.assert_array_equal(got, ref)
    st = oracle.tri_stats(got)
    f = got.ravel().astype(np.int64)
    assert st[0] == f.sum() and st[1] == sum(f[a] * f[b] for a, b in bl)


def test_three_by_three_enumeration():
    L, beta, J, h = 3, 0.3, 1.0, 0.05
    bl = bonds(L)
    Z = E1 = M2 = 0.0
    for bits in itertools.product([-1, 1], repeat=L * L):
        s = np.array(bits, dtype=np.int64).reshape(L, L)
        e = energy(s, J, h, bl)
        w = math.exp(-beta * e)
        Z += w
        E1 += w * e
        M2 += w * s.sum() ** 2
    exact_E, exact_M2 = E1 / Z, M2 / Z
    Es, M2s = [], []
    for lat in range(64):
        s = oracle.init_ising(L, SEED, lat)
        st = oracle.tri_run(s, beta, J, h, SEED, lat, 0, 600)[100:]
        Es.append(-J * st[:, 1] - h * st[:, 0])
        M2s.append(st[:, 0].astype(np.float64) ** 2)
    Es, M2s = np.concatenate(Es), np.concatenate(M2s)
    assert abs(Es.mean() - exact_E) < 5 * binned_stderr(Es) + 1e-9, (Es.mean(), exact_E)
    assert abs(M2s.mean() - exact_M2) < 5 * binned_stderr(M2s) + 1e-9, (M2s.mean(), exact_M2)

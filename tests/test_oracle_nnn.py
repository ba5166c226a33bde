"""Pins of the first-and-second-neighbour Ising oracle (other orders of
neighbourhood, Sec. "Ising model"; H = -J sum_nn s s - J2 sum_diag s s - h sum s):
a bit-exact replica whose energy change is a brute-force difference of the
Hamiltonian over an independently built eight-neighbour bond list, the
(M, B, B2) statistics recounted from that list, the four-colour rule, exact
enumeration of the 4 x 4 periodic lattice (2^16 states) against chain
averages (with J2 = 0 against the plain square-lattice enumeration), and the
fluctuation estimator of d<E>/dJ2 against a finite difference of the exact
expectation."""
import math

import numpy as np

import oracle
from oracle import estimator
from tests.exact import binned_stderr, ising_exact

SEED = 0x5EC0DD

NN = [(1, 0), (-1, 0), (0, 1), (0, -1)]
DIAG = [(1, 1), (1, -1), (-1, 1), (-1, -1)]


def bonds(L, dirs):
    """Each unordered pair (site, site + d) for d in dirs once."""
    out = set()
    for y in range(L):
        for x in range(L):
            for dx, dy in dirs:
                a, b = y * L + x, ((y + dy) % L) * L + (x + dx) % L
                out.add((min(a, b), max(a, b)))
    return sorted(out)


def bond_sum(s, bl):
    f = s.ravel().astype(np.int64)
    return int(sum(f[a] * f[b] for a, b in bl))


def energy(s, J, J2, h, b1, b2):
    return -J * bond_sum(s, b1) - J2 * bond_sum(s, b2) - h * int(s.sum())


def test_bond_lists_and_colours():
    L = 8
    b1, b2 = bonds(L, NN), bonds(L, DIAG)
    assert len(b1) == 2 * L * L and len(b2) == 2 * L * L
    colour = lambda i: ((i % L) & 1) | (((i // L) & 1) << 1)
    # no bond of either order joins two sites of one colour
    assert all(colour(a) != colour(b) for a, b in b1 + b2)


def test_replica_with_brute_force_energy_change():
    L, beta, J, J2, h = 8, 0.45, 1.0, -0.6, 0.15
    b1, b2 = bonds(L, NN), bonds(L, DIAG)
    s0 = oracle.init_ising(L, SEED, 5)
    got = s0.copy()
    for t in range(3):
        oracle.nnn_sweep(got, beta, J, J2, h, SEED, 5, t)
    ref = s0.copy()
    key = [SEED & 0xFFFFFFFF, SEED >> 32]
    flips = 0
    for t in range(3):
        for c in range(4):
            for y in range(L):
                for x in range(L):
                    if ((x & 1) | ((y & 1) << 1)) != c:
                        continue
                    flipped = ref.copy()
                    flipped[y, x] = -flipped[y, x]
                    dE = float(energy(flipped, J, J2, h, b1, b2) - energy(ref, J, J2, h, b1, b2))
                    k = (y >> 1) * (L // 2) + (x >> 1)
                    u = int(oracle.philox4x32_10([k >> 2, 5, t, c], key)[k & 3])
                    if dE <= 0 or u < oracle.accept_count(beta, dE):
                        ref = flipped
                        flips += 1
    assert flips > 20
    np.testing.assert_array_equal(got, ref)
    st = oracle.nnn_stats(got)
    assert st[0] == int(got.sum()) and st[1] == bond_sum(got, b1) and st[2] == bond_sum(got, b2)


def test_sweep_is_the_four_substeps_in_order():
    L = 12
    s = oracle.init_ising(L, SEED, 1)
    a, b = s.copy(), s.copy()
    oracle.nnn_sweep(a, 0.3, 0.8, 0.4, -0.1, SEED, 1, 7)
    for c in range(4):
        oracle.nnn_substep(b, 0.3, 0.8, 0.4, -0.1, SEED, 1, 7, c)
    np.testing.assert_array_equal(a, b)
    # a different colour order gives a different chain (the order is part of the rule)
    d = s.copy()
    for c in (1, 0, 3, 2):
        oracle.nnn_substep(d, 0.3, 0.8, 0.4, -0.1, SEED, 1, 7, c)
    assert not np.array_equal(a, d)


def enum_4x4():
    L = 4
    n = L * L
    idx = np.arange(2 ** n, dtype=np.int64)
    s = (1 - 2 * ((idx[:, None] >> np.arange(n)) & 1)).reshape(-1, L, L)
    M = s.sum(axis=(1, 2))
    B = (s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) + (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    diag1 = np.roll(np.roll(s, -1, axis=1), -1, axis=2)   # (x+1, y+1)
    diag2 = np.roll(np.roll(s, 1, axis=1), -1, axis=2)    # (x+1, y-1)
    B2 = (s * diag1).sum(axis=(1, 2)) + (s * diag2).sum(axis=(1, 2))
    return M.astype(np.float64), B.astype(np.float64), B2.astype(np.float64)


def exact(beta, J, J2, h):
    M, B, B2 = enum_4x4()
    E = -J * B - J2 * B2 - h * M
    lw = -beta * E
    w = np.exp(lw - lw.max())
    w /= w.sum()
    return {"E": float(w @ E), "M2": float(w @ (M * M)), "B2": float(w @ B2)}


def chain(beta, J, J2, h, n_lat=48, sweeps=1500, burn=100):
    out = []
    for lat in range(n_lat):
        s = oracle.init_ising(4, SEED, lat)
        out.append(oracle.nnn_run(s, beta, J, J2, h, SEED, lat, 0, sweeps)[burn:])
    return np.concatenate(out).astype(np.float64)


def test_four_by_four_enumeration():
    for beta, J, J2, h in [(0.4, 1.0, -0.5, 0.1), (0.3, 0.5, 0.7, 0.0)]:
        ex = exact(beta, J, J2, h)
        st = chain(beta, J, J2, h)
        E = -J * st[:, 1] - J2 * st[:, 2] - h * st[:, 0]
        for got, want in ((E, ex["E"]), (st[:, 0] ** 2, ex["M2"]), (st[:, 2], ex["B2"])):
            assert abs(got.mean() - want) < 5 * binned_stderr(got) + 1e-9, (got.mean(), want)


def test_without_diagonal_coupling_the_law_is_the_square_lattice_one():
    beta, J, h = 0.35, 1.0, 0.05
    ref = ising_exact(beta, J, h, 4)
    mine = exact(beta, J, 0.0, h)
    assert abs(mine["E"] - ref["E"]) < 1e-9 and abs(mine["M2"] - ref["M2"]) < 1e-9
    st = chain(beta, J, 0.0, h)
    E = -J * st[:, 1] - h * st[:, 0]
    assert abs(E.mean() - ref["E"]) < 5 * binned_stderr(E)


def test_estimator_matches_the_exact_derivative():
    beta, J, J2, h = 0.3, 1.0, -0.4, 0.1
    d = 1e-5
    fd = (exact(beta, J, J2 + d, h)["E"] - exact(beta, J, J2 - d, h)["E"]) / (2 * d) / 16.0
    fdJ = (exact(beta, J + d, J2, h)["E"] - exact(beta, J - d, J2, h)["E"]) / (2 * d) / 16.0
    st = chain(beta, J, J2, h, n_lat=64, sweeps=2000)
    gr = estimator.nnn_grad(st[None], beta, J, J2, h, 16.0)
    # statistical: the covariance estimate from ~1.2e5 correlated samples
    for g, want in ((gr[("E", "J2")], fd), (gr[("E", "J")], fdJ)):
        assert math.isfinite(g)
        assert abs(g - want) < 0.05 * abs(want) + 0.01, (g, want)

"""Pins for the oracle's Ising chain: exact enumeration, Onsager/Yang,
detailed balance and an independent brute-force replica (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from tests import exact


def _replica_ising_sweep(s, beta, J, h, seed, lat, t):
    """One sweep written from the definitions: for every site of colour 0,
    then colour 1, dE = H(flipped) - H(current) from the full Hamiltonian."""
    L = s.shape[0]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    b = float(np.float32(beta))
    Jd, hd = float(np.float32(J)), float(np.float32(h))
    for c in (0, 1):
        for y in range(L):
            for x in range(L):
                if (x + y) & 1 != c:
                    continue
                E0 = exact.ising_H(s, Jd, hd)
                s[y, x] = -s[y, x]
                E1 = exact.ising_H(s, Jd, hd)
                s[y, x] = -s[y, x]
                k = (y * L + x) >> 1
                u = int(oracle.philox4x32_10([k >> 2, lat, t, c], key)[k & 3])
                dE = E1 - E0
                if dE <= 0:
                    acc = True
                else:
                    acc = u < max(math.floor(math.exp(-b * dE) * 2.0 ** 32), 1)
                if acc:
                    s[y, x] = -s[y, x]


@pytest.mark.parametrize("L,beta,J,h", [(8, 0.4, 1.0, 0.25), (6, 0.7, -1.0, 0.0), (4, 0.3, 0.5, -0.5)])
def test_ising_sweep_matches_bruteforce_replica(L, beta, J, h):
    seed, lat = 0xDEADBEEF12345, 5
    s = oracle.init_ising(L, seed, lat).copy()
    r = s.copy()
    for t in range(3):
        oracle.ising_sweep(s, beta, J, h, seed, lat, 7 + t)
        _replica_ising_sweep(r, beta, J, h, seed, lat, 7 + t)
        assert np.array_equal(s, r)


def test_ising_init_uses_documented_draws():
    L, seed, lat = 8, 99, 3
    s = oracle.init_ising(L, seed, lat)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(L * L):
        u = int(oracle.philox4x32_10([i >> 2, lat, 0xFFFFFFFF, 0], key)[i & 3])
        assert s.flat[i] == (1 if u >> 31 else -1)
    # A random start is roughly balanced.
    assert abs(int(oracle.init_ising(64, 0, 0).sum())) < 4 * 64


def test_ising_stats_definition():
    rng = np.random.default_rng(1)
    for L in (4, 6, 10):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L))
        M, B = oracle.ising_stats(s)
        assert M == int(s.sum())
        assert B == -int(exact.ising_H(s, 1.0, 0.0))


def test_detailed_balance_of_colour_substep_4x4():
    """Every single-site factor of a colour sub-step is reversible w.r.t.
    exp(-beta H); hence so is the sub-step.  dE from the Hamiltonian."""
    L = 4
    M, B = exact.ising_4x4_MB(L)
    for beta, J, h in [(0.44, 1.0, 0.0), (0.3, 1.0, 0.3), (0.8, -0.7, 0.1)]:
        E = -J * B.astype(np.float64) - h * M.astype(np.float64)
        rng = np.random.default_rng(0)
        for x in rng.integers(0, 2 ** 16, size=200):
            for i in range(16):
                xi = x ^ (1 << i)
                dE = E[xi] - E[x]
                p_fwd = oracle.accept_count(beta, dE) / 2.0 ** 32
                p_bwd = oracle.accept_count(beta, -dE) / 2.0 ** 32
                lhs = math.exp(-beta * E[x]) * p_fwd
                rhs = math.exp(-beta * E[xi]) * p_bwd
                assert abs(lhs - rhs) <= 2.0 ** -31 * max(lhs, rhs) / min(p_fwd, p_bwd) + 1e-300


@pytest.mark.parametrize("beta,J,h", [(0.3, 1.0, 0.0), (0.44, 1.0, 0.0), (0.6, 1.0, 0.2), (0.5, -1.0, 0.0)])
def test_ising_4x4_matches_exact_enumeration(beta, J, h):
    L, n = 4, 60000
    s = oracle.init_ising(L, 7, 0).copy()
    oracle.ising_run(s, beta, J, h, 7, 0, 0, 500, record=False)
    st = oracle.ising_run(s, beta, J, h, 7, 0, 500, n)
    M = st[:, 0].astype(np.float64)
    B = st[:, 1].astype(np.float64)
    E = -J * B - h * M
    ex = exact.ising_exact(beta, J, h, L)
    for name, series, want in [("E", E, ex["E"]), ("M2", M * M, ex["M2"]), ("absM", np.abs(M), ex["absM"])]:
        err = exact.binned_stderr(series, 50)
        assert abs(series.mean() - want) < 5 * err + 1e-9, (name, series.mean(), want, err)


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_large_lattice_matches_onsager(beta):
    L = 96
    s = oracle.init_ising(L, 11, 2).copy()
    if beta > exact.BETA_C_ISING:
        # A random start coarsens into long-lived stripes at low temperature;
        # start in one of the two ordered states instead.
        s[:] = 1
    oracle.ising_run(s, beta, 1.0, 0.0, 11, 2, 0, 400, record=False)
    st = oracle.ising_run(s, beta, 1.0, 0.0, 11, 2, 400, 2000)
    N = L * L
    e = -st[:, 1].astype(np.float64) / N
    m = np.abs(st[:, 0].astype(np.float64)) / N
    u = exact.onsager_u(beta)
    assert abs(e.mean() - u) < 5 * exact.binned_stderr(e) + 2e-3, (e.mean(), u)
    if beta > exact.BETA_C_ISING:
        assert abs(m.mean() - exact.yang_m(beta)) < 5 * exact.binned_stderr(m) + 2e-3
    else:
        assert m.mean() < 0.05


def test_onsager_closed_form_limits():
    # Ground state: two satisfied bonds per site; infinite temperature: 0.
    assert abs(exact.onsager_u(20.0) + 2.0) < 1e-9
    assert abs(exact.onsager_u(1e-4)) < 1e-3
    # High-temperature series (closed loops of 4 and 6 bonds on the square
    # lattice): u = -2v - 4v^3 - 8v^5 + O(v^7), v = tanh(K).
    K = 0.05
    v = math.tanh(K)
    assert abs(exact.onsager_u(K) + 2 * v + 4 * v ** 3 + 8 * v ** 5) < 1e-7

"""Pins for the oracle's q-state Potts chain (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from tests import exact


def _replica_potts_sweep(s, q, beta, J, seed, lat, t):
    """One sweep from the definitions: proposal among the q-1 other values,
    dE from the full Hamiltonian H = -J sum delta, Metropolis with 2^-32 draws."""
    L = s.shape[0]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    b = float(np.float32(beta))
    Jd = float(np.float32(J))
    for c in (0, 1):
        for y in range(L):
            for x in range(L):
                if (x + y) & 1 != c:
                    continue
                k = (y * L + x) >> 1
                r = oracle.philox4x32_10([k >> 1, lat, t, c], key)
                u0, u1 = int(r[2 * (k & 1)]), int(r[2 * (k & 1) + 1])
                old = int(s[y, x])
                new = (old + 1 + ((u1 * (q - 1)) >> 32)) % q
                assert new != old
                E0 = exact.potts_H(s, Jd)
                s[y, x] = new
                E1 = exact.potts_H(s, Jd)
                s[y, x] = old
                dE = E1 - E0
                acc = dE <= 0 or u0 < max(math.floor(math.exp(-b * dE) * 2.0 ** 32), 1)
                if acc:
                    s[y, x] = new


@pytest.mark.parametrize("L,q,beta,J", [(8, 3, 1.0, 1.0), (6, 8, 1.2, 1.0), (4, 2, 0.5, -1.0), (8, 5, 0.9, 0.75)])
def test_potts_sweep_matches_bruteforce_replica(L, q, beta, J):
    seed, lat = 4242, 9
    s = oracle.init_potts(L, q, seed, lat).copy()
    r = s.copy()
    for t in range(3):
        oracle.potts_sweep(s, q, beta, J, seed, lat, t)
        _replica_potts_sweep(r, q, beta, J, seed, lat, t)
        assert np.array_equal(s, r)


def test_potts_init_and_stats():
    L, q = 16, 8
    s = oracle.init_potts(L, q, 5, 1)
    assert s.max() < q
    st = oracle.potts_stats(s, q)
    assert st[0] == -int(exact.potts_H(s, 1.0))
    assert list(st[1:]) == [int((s == k).sum()) for k in range(q)]


def test_potts_q2_is_ising_with_half_coupling():
    """H_Potts(q=2, J) = -(J/2) sum s s' - const: the q=2 chain samples the
    Ising law with J/2.  Compare <E_Ising> on 4x4 with exact enumeration."""
    L, Jp, beta = 4, 2.0, 0.5
    s = oracle.init_potts(L, 2, 3, 0).copy()
    oracle.potts_run(s, 2, beta, Jp, 3, 0, 0, 500, record=False)
    st = oracle.potts_run(s, 2, beta, Jp, 3, 0, 500, 60000)
    Beq = st[:, 0].astype(np.float64)
    B_ising = 2.0 * Beq - 2 * L * L          # equal bond +1, unequal -1
    ex = exact.ising_exact(beta, Jp / 2.0, 0.0, L)
    err = exact.binned_stderr(B_ising, 50)
    assert abs(B_ising.mean() - ex["B"]) < 5 * err, (B_ising.mean(), ex["B"], err)


@pytest.fixture(scope="module")
def potts3_hist():
    return exact.potts_4x4_hist(3, 4)


def test_potts_exact_histogram_counts(potts3_hist):
    assert potts3_hist.sum() == 3 ** 16
    # All-equal states: 3 of them with all 32 bonds equal.
    assert potts3_hist[32].sum() == 3


@pytest.mark.parametrize("beta", [0.6, math.log(1 + math.sqrt(3)), 1.4])
def test_potts_q3_4x4_matches_exact_enumeration(potts3_hist, beta):
    L, q, J = 4, 3, 1.0
    s = oracle.init_potts(L, q, 17, 0).copy()
    oracle.potts_run(s, q, beta, J, 17, 0, 0, 500, record=False)
    st = oracle.potts_run(s, q, beta, J, 17, 0, 500, 60000)
    E = -J * st[:, 0].astype(np.float64)
    Mq = (q * st[:, 1:].max(axis=1).astype(np.float64) - L * L) / (q - 1)
    ex = exact.potts_exact(potts3_hist, beta, J, q, L)
    assert abs(E.mean() - ex["E"]) < 5 * exact.binned_stderr(E, 50), (E.mean(), ex["E"])
    assert abs(Mq.mean() - ex["Mq"]) < 5 * exact.binned_stderr(Mq, 50), (Mq.mean(), ex["Mq"])


def test_potts_q3_ordering_across_beta_c():
    """Order parameter grows through beta_c = ln(1 + sqrt(q)) (q=3, L=32)."""
    L, q = 32, 3
    bc = math.log(1 + math.sqrt(q))
    ms = []
    for f in (0.8, 1.25):
        s = oracle.init_potts(L, q, 1, 0).copy()
        oracle.potts_run(s, q, bc * f, 1.0, 1, 0, 0, 600, record=False)
        st = oracle.potts_run(s, q, bc * f, 1.0, 1, 0, 600, 400)
        ms.append(((q * st[:, 1:].max(axis=1) - L * L) / (q - 1) / (L * L)).mean())
    assert ms[0] < 0.25 < 0.75 < ms[1]

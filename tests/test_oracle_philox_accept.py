"""Pins for the oracle's random stream and acceptance rule (CPU only)."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    got = oracle.philox4x32_10(ctr, key)
    assert [int(x) for x in got] == want


def test_philox_counter_words_all_matter():
    base = oracle.philox4x32_10([5, 6, 7, 8], [9, 10])
    for i in range(4):
        c = [5, 6, 7, 8]
        c[i] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(c, [9, 10]), base)
    for i in range(2):
        k = [9, 10]
        k[i] ^= 1
        assert not np.array_equal(oracle.philox4x32_10([5, 6, 7, 8], k), base)


def test_philox_uniform_chi2():
    # 4 * 4096 outputs, top 4 bits into 16 bins: chi^2 with 15 dof.
    vals = np.concatenate([oracle.philox4x32_10([g, 3, 11, 1], [0x1234, 0x5678]) for g in range(4096)])
    counts = np.bincount((vals >> 28).astype(np.int64), minlength=16)
    exp = len(vals) / 16
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 40.0  # p ~ 5e-4 for 15 dof


def test_accept_count_special_cases():
    two32 = 4294967296.0
    # Downhill and flat moves are always accepted.
    assert oracle.accept_count(0.7, -3.0) == two32
    assert oracle.accept_count(0.7, 0.0) == two32
    # Infinite temperature accepts everything.
    assert oracle.accept_count(0.0, 8.0) == two32
    # The floor keeps every move reachable: p < 2^-32 still accepts one value.
    assert oracle.accept_count(50.0, 8.0) == 1.0
    # Monotone in beta * dE and strictly between for moderate values.
    a = [oracle.accept_count(b, 4.0) for b in (0.1, 0.2, 0.4, 0.8)]
    assert all(x > y for x, y in zip(a, a[1:]))
    assert 0 < a[-1] < two32


@pytest.mark.parametrize("beta", [0.2, 0.44, 0.9])
@pytest.mark.parametrize("dE", [0.5, 4.0, 8.0])
def test_accept_detailed_balance_pair(beta, dE):
    """p(dE) / p(-dE) = exp(-beta dE) up to the 2^-32 quantisation (Alg. 1)."""
    p_up = oracle.accept_count(beta, dE) / 4294967296.0
    p_down = oracle.accept_count(beta, -dE) / 4294967296.0
    ratio = p_up / p_down
    want = math.exp(-beta * dE)
    assert abs(ratio - want) <= 2.0 ** -32 + 1e-15


def test_accept_decision_matches_count():
    for beta, dE in [(0.4, 4.0), (0.6, 8.0), (0.3, 2.5)]:
        k = int(oracle.accept_count(beta, dE))
        assert oracle.lib().or_accept(beta, dE, k - 1) == 1
        assert oracle.lib().or_accept(beta, dE, k) == 0


@pytest.mark.parametrize("g0,n", [(0, 0), (0, 1), (12345, 517), (2**32 - 300, 300)])
def test_philox_xor_digest_equals_the_blocks_it_covers(g0, n):
    """The stream digest (XOR of every word of blocks g0 .. g0 + n - 1) equals
    the XOR of the known-answer-pinned single blocks, in any order."""
    seed, lat, t, c = 0x0123456789ABCDEF, 7, 99, 1
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = 0
    for g in range(g0, g0 + n):
        r = oracle.philox4x32_10([g, lat, t, c], key)
        want ^= int(r[0]) ^ int(r[1]) ^ int(r[2]) ^ int(r[3])
    assert oracle.philox_xor(seed, lat, t, c, g0, n) == want
    if n > 1:   # a split range XORs to the whole
        h = n // 2
        assert oracle.philox_xor(seed, lat, t, c, g0, h) ^ oracle.philox_xor(seed, lat, t, c, g0 + h, n - h) == want

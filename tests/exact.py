"""Exact results used to pin the oracle (test helper, no method code).

* Exhaustive enumeration of the 4x4 periodic Ising lattice (2^16 states) and
  of the 4x4 periodic q=3 Potts lattice (3^16 states, enumerated row by row).
* Onsager's exact internal energy and Yang's spontaneous magnetisation of the
  infinite square-lattice Ising model (H = -J sum_<ij> s_i s_j).
* The Boltzmann energy H(s) written from the Hamiltonians, for brute-force
  energy differences.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


# ----------------------------------------------------------------------------
# Hamiltonians written directly from their definitions (bonds counted once).
# ----------------------------------------------------------------------------
def ising_H(s, J, h):
    s = np.asarray(s, dtype=np.float64)
    bonds = (s * np.roll(s, -1, axis=1)).sum() + (s * np.roll(s, -1, axis=0)).sum()
    return -J * bonds - h * s.sum()


def potts_H(s, J):
    s = np.asarray(s)
    eq = (s == np.roll(s, -1, axis=1)).sum() + (s == np.roll(s, -1, axis=0)).sum()
    return -J * float(eq)


MOORE_HALF = ((1, 0), (-1, 1), (0, 1), (1, 1))  # (dx, dy): each unordered pair once


def cpm_adhesion(ids, types, Jtab):
    ids = np.asarray(ids)
    E = 0
    for dx, dy in MOORE_HALF:
        nb = np.roll(np.roll(ids, -dy, axis=0), -dx, axis=1)
        diff = ids != nb
        E += int(np.asarray(Jtab)[types[ids], types[nb]][diff].sum())
    return E


# ----------------------------------------------------------------------------
# 4x4 Ising enumeration
# ----------------------------------------------------------------------------
_ISING_CACHE = {}


def ising_4x4_MB(L=4):
    """(M, B) for all 2^(L*L) states."""
    if L in _ISING_CACHE:
        return _ISING_CACHE[L]
    n = L * L
    idx = np.arange(2 ** n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n)) & 1
    s = (1 - 2 * bits).astype(np.int64).reshape(-1, L, L)
    M = s.sum(axis=(1, 2))
    B = (s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) + (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    _ISING_CACHE[L] = (M, B)
    return M, B


def ising_exact(beta, J, h, L=4):
    """Exact expectations over the Boltzmann law of the LxL periodic lattice."""
    M, B = ising_4x4_MB(L)
    M = M.astype(np.float64)
    B = B.astype(np.float64)
    E = -J * B - h * M
    logw = -beta * E
    w = np.exp(logw - logw.max())
    w /= w.sum()
    N = L * L
    ex = lambda f: float(np.sum(w * f))
    return {
        "E": ex(E), "M": ex(M), "absM": ex(np.abs(M)), "M2": ex(M * M), "E2": ex(E * E),
        "B": ex(B), "B2": ex(B * B), "MB": ex(M * B), "N": N,
        "w": w, "Mall": M, "Ball": B,
    }


def ising_exact_grad(beta, J, h, L=4):
    """Exact d<O>/dtheta from the fluctuation identity over the enumeration."""
    ex = ising_exact(beta, J, h, L)
    w, M, B, N = ex["w"], ex["Mall"], ex["Ball"], ex["N"]
    E = -J * B - h * M
    mean = lambda f: float(np.sum(w * f))
    cov = lambda a, b: mean(a * b) - mean(a) * mean(b)
    return {
        ("E", "J"): mean(-B / N) - beta * cov(E / N, -B),
        ("E", "h"): mean(-M / N) - beta * cov(E / N, -M),
        ("M", "J"): -beta * cov(M / N, -B),
        ("M", "h"): -beta * cov(M / N, -M),
    }


# ----------------------------------------------------------------------------
# 4x4 q-state Potts enumeration (row transfer, exhaustive)
# ----------------------------------------------------------------------------
def potts_4x4_hist(q=3, L=4):
    """hist[Beq, nmax]: number of states with Beq equal bonds and max_k n_k = nmax."""
    rows = np.array(list(itertools.product(range(q), repeat=L)), dtype=np.int64)
    R = rows.shape[0]
    h_eq = (rows == np.roll(rows, -1, axis=1)).sum(axis=1)
    v_eq = (rows[:, None, :] == rows[None, :, :]).sum(axis=2)
    cnt = np.stack([(rows == k).sum(axis=1) for k in range(q)], axis=1)
    nb = 2 * L * L
    hist = np.zeros((nb + 1, L * L + 1), dtype=np.int64)
    r1, r2, r3 = np.meshgrid(np.arange(R), np.arange(R), np.arange(R), indexing="ij")
    r1 = r1.ravel(); r2 = r2.ravel(); r3 = r3.ravel()
    inner = h_eq[r1] + h_eq[r2] + h_eq[r3] + v_eq[r1, r2] + v_eq[r2, r3]
    c123 = cnt[r1] + cnt[r2] + cnt[r3]
    for r0 in range(R):
        Beq = inner + h_eq[r0] + v_eq[r0, r1] + v_eq[r3, r0]
        nmax = (c123 + cnt[r0]).max(axis=1)
        np.add.at(hist, (Beq, nmax), 1)
    return hist


def potts_exact(hist, beta, J, q=3, L=4):
    N = L * L
    Beq = np.arange(hist.shape[0], dtype=np.float64)[:, None]
    nmax = np.arange(hist.shape[1], dtype=np.float64)[None, :]
    logw = beta * J * Beq + np.log(np.maximum(hist, 1)) * (hist > 0)
    logw = np.where(hist > 0, logw, -np.inf)
    w = np.exp(logw - logw.max())
    w /= w.sum()
    Mq = (q * nmax - N) / (q - 1)
    return {"E": float(np.sum(w * (-J * Beq))), "B": float(np.sum(w * Beq + 0 * nmax)),
            "Mq": float(np.sum(w * Mq)), "N": N}


# ----------------------------------------------------------------------------
# Onsager / Yang
# ----------------------------------------------------------------------------
def _agm(a, b):
    for _ in range(60):
        a, b = 0.5 * (a + b), math.sqrt(a * b)
    return a


def ellipk(k):
    """Complete elliptic integral of the first kind, modulus k (via the AGM)."""
    return math.pi / (2.0 * _agm(1.0, math.sqrt(1.0 - k * k)))


def onsager_u(beta, J=1.0):
    """Internal energy per site of the infinite 2D Ising model."""
    K = beta * J
    k = 2.0 * math.sinh(2 * K) / math.cosh(2 * K) ** 2
    return -J / math.tanh(2 * K) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(2 * K) ** 2 - 1.0) * ellipk(k))


BETA_C_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))


def yang_m(beta, J=1.0):
    """Spontaneous magnetisation per site (0 above the critical temperature)."""
    if beta * J <= BETA_C_ISING:
        return 0.0
    return (1.0 - math.sinh(2 * beta * J) ** -4) ** 0.125


def binned_stderr(x, nbins=20):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbins
    means = x[: n * nbins].reshape(nbins, n).mean(axis=1)
    return float(means.std(ddof=1) / math.sqrt(nbins))

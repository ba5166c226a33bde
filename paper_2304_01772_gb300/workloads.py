"""Seeded synthetic workloads: lattice sizes, temperatures, couplings and
fields for the benchmark configurations and the tests.

This module draws inputs only; it holds none of the Monte Carlo arithmetic.
Random draws come from a self-contained splitmix64 generator so that the same
seed gives the same workload on every machine and numpy version.

Configurations (sizes and parameter ranges of the paper's workloads, Sec.
"Results", and of the five benchmark cases):
  ising_small    8 Ising lattices 64x64, beta = linspace(0.2, 0.6, 8), J=1, h=0
  potts_batch    64 q-state Potts lattices 1024x1024, beta = beta_c(q) * linspace(0.8, 1.2, 64)
  uneven512      512 Ising lattices, L = 2^e with e uniform in {5..11},
                 beta ~ U(0.3, 0.55), h ~ N(0, 0.05)
  fit256         128 Ising chains 256x256 at beta = 0.45
  nnn256         256 Ising lattices 256x256 with first and second neighbours:
                 J = 1, J2 ~ U(-0.5, 0.5), beta ~ U(0.2, 0.45), h ~ N(0, 0.05)
  cpm1024        cellular Potts 1024x1024, 2000 cells of 20x20 in 50 columns,
                 J = [[0,16,16],[16,2,11],[16,11,14]], A = 400, lambda = 1, T = 10
"""
from __future__ import annotations

import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """Steele, Lea & Flood (2014) splitmix64 stream."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def integer(self, lo: int, hi: int) -> int:
        """Uniform in [lo, hi] (inclusive)."""
        return lo + self.next_u64() % (hi - lo + 1)

    def normal(self) -> float:
        u1 = max(self.uniform(), 1e-300)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def linspace(a, b, n):
    return [a + (b - a) * i / (n - 1) for i in range(n)] if n > 1 else [a]


def potts_beta_c(q: int) -> float:
    """Critical coupling ln(1 + sqrt(q)) of the square-lattice Potts model."""
    return math.log(1.0 + math.sqrt(q))


def ising_small(n=8, L=64):
    return [dict(L=L, beta=b, J=1.0, h=0.0) for b in linspace(0.2, 0.6, n)]


def potts_batch(q=3, n=64, L=1024):
    bc = potts_beta_c(q)
    return [dict(L=L, q=q, beta=bc * f, J=1.0, h=0.0) for f in linspace(0.8, 1.2, n)]


def uneven512(n=512, seed=0, emin=5, emax=11):
    r = SplitMix64(seed)
    out = []
    for _ in range(n):
        e = r.integer(emin, emax)
        beta = 0.3 + 0.25 * r.uniform()
        h = 0.05 * r.normal()
        out.append(dict(L=1 << e, beta=beta, J=1.0, h=h))
    return out


def nnn256(n=256, L=256, seed=0):
    r = SplitMix64(seed)
    out = []
    for _ in range(n):
        beta = 0.2 + 0.25 * r.uniform()
        J2 = -0.5 + r.uniform()
        h = 0.05 * r.normal()
        out.append(dict(L=L, beta=beta, J=1.0, J2=J2, h=h, geometry=2))
    return out


def fit256(n=128, L=256, beta=0.45, J=1.0, h=0.0):
    return [dict(L=L, beta=beta, J=J, h=h) for _ in range(n)]


CPM_J = [[0, 16, 16], [16, 2, 11], [16, 11, 14]]


def cpm1024():
    return dict(L=1024, J=CPM_J, lam=1, target=400, n_cells=2000, T=10.0, side=20, cols=50)


def cpm_paper():
    """The paper's cell-sorting setup: 36 cells + medium, A = 25, T = 8 (Sec. "Results")."""
    return dict(L=64, J=CPM_J, lam=1, target=25, n_cells=36, T=8.0, side=5, cols=6)


def site_count(lattices):
    return sum(d["L"] * d["L"] for d in lattices)

"""Differentiable Monte Carlo (Alg. 2) -- TEST INFRASTRUCTURE ONLY.

Thin numpy wrappers around the plain C restatement in ``spin_oracle.c``
(float64 throughout): the relaxed Ising sub-step with one coupling per bond,
its hand-written reverse pass, the L2 pattern loss of Sec. "Optimization of
the exchange parameters" and the final discretisation.  Arrays: spins and
targets [L, L]; couplings J [2, L, L] with J[0] the bond to the right neighbour
and J[1] the bond to the neighbour below (periodic).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _p, lib

_D = ctypes.c_double


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def substep(s, J, beta, h, alpha, seed, lattice, sweep, colour):
    """One colour sub-step in place (s float64 [L, L])."""
    L = s.shape[0]
    J = _c(J)
    lib().or_dmc_substep(L, _p(J[0], _D), _p(J[1], _D), beta, h, alpha, seed, lattice, sweep, colour,
                         _p(s, _D))


def run(s, J, beta, h, alpha, seed, lattice, sweep0, n_sweeps, tape=False):
    """n_sweeps sweeps in place; with tape=True returns the states before each
    of the 2 n_sweeps sub-steps, [2 n_sweeps, L, L]."""
    L = s.shape[0]
    J = _c(J)
    tp = np.zeros((2 * n_sweeps, L, L)) if tape else None
    lib().or_dmc_run(L, _p(J[0], _D), _p(J[1], _D), beta, h, alpha, seed, lattice, sweep0, n_sweeps,
                     _p(s, _D), _p(tp, _D) if tape else None)
    return tp


def backward(tape, J, g_final, beta, h, alpha, seed, lattice, sweep0):
    """Reverse pass: returns (dL/ds before the first sub-step, dL/dJ [2, L, L])."""
    n_sub, L, _ = tape.shape
    J = _c(J)
    g = _c(g_final).copy()
    gJ = np.zeros((2, L, L))
    lib().or_dmc_backward(L, _p(J[0], _D), _p(J[1], _D), beta, h, alpha, seed, lattice, sweep0,
                          n_sub // 2, _p(_c(tape), _D), _p(g, _D), _p(gJ[0], _D), _p(gJ[1], _D))
    return g, gJ


def loss(s, target):
    """(sum (target - s)^2, dL/ds)."""
    g = np.zeros_like(_c(s))
    v = lib().or_dmc_loss(s.shape[0], _p(_c(s), _D), _p(_c(target), _D), _p(g, _D))
    return float(v), g


def discretize(s):
    out = _c(s).copy()
    lib().or_dmc_discretize(out.size, _p(out, _D))
    return out


def energy(s, J, h):
    """(E, dE/ds) of relaxed spins under per-bond couplings."""
    L = s.shape[0]
    J = _c(J)
    g = np.zeros((L, L))
    E = lib().or_dmc_energy(L, _p(J[0], _D), _p(J[1], _D), h, _p(_c(s), _D), _p(g, _D))
    return float(E), g


def spin_step(s, g, eta):
    """s <- clip(s - eta sign(g), -1, 1), returned as a new array."""
    out = _c(s).copy()
    lib().or_dmc_spin_step(out.size, _p(out, _D), _p(_c(g), _D), eta)
    return out


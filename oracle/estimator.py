"""Fluctuation (score-function) estimator of d<O>/dtheta -- TEST INFRASTRUCTURE ONLY.

For a Boltzmann law pi(x) = exp(-beta H(x; theta)) / Z the derivative of an
expectation is

    d<O>/dtheta = <dO/dtheta> - beta * ( <O dH/dtheta> - <O><dH/dtheta> ),

i.e. the explicit term plus -beta times the covariance of O with dH/dtheta.
The paper differentiates through relaxed Monte Carlo steps instead (Alg. 2);
this estimator is the plain statistical-mechanics identity, written out here
in float64 with the two-pass covariance, over samples t >= burn_in pooled
over every chain given (chains that share theta).

Ising (H = -J sum s s - h sum s):  dH/dJ = -B, dH/dh = -M, with per-sample
integers M = sum s and B = sum over bonds s s'.  O is E/N (E = -J B - h M,
so dO/dJ = -B/N, dO/dh = -M/N) or M/N (no explicit term).

Cellular Potts (Eq. "h"): dH/dJ_ab = C_ab (contacts between cell types a<=b),
dH/dlambda = sum_cells (a-A)^2, dH/dA = -2 lambda sum_cells (a-A); beta = 1/T.
O is the adhesion energy per site, sum_{a<=b} J_ab C_ab / N.
"""
from __future__ import annotations

import numpy as np


def _cov(o: np.ndarray, d: np.ndarray) -> float:
    o = np.asarray(o, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    return float(np.mean((o - o.mean()) * (d - d.mean())))


def fluctuation_grad(O, dO, dH, beta):
    """<dO> - beta * Cov(O, dH) for one parameter (arrays over samples)."""
    O = np.asarray(O, dtype=np.float64)
    explicit = 0.0 if dO is None else float(np.mean(np.asarray(dO, dtype=np.float64)))
    return explicit - float(beta) * _cov(O, dH)


def ising_grad(stats, beta, J, h, N, burn_in=0):
    """stats: [..., T, 2] integer (M, B) per sweep; leading axes are pooled chains.

    Returns {('E','J'), ('E','h'), ('M','J'), ('M','h')} -> float.
    """
    st = np.asarray(stats)
    st = st.reshape(-1, st.shape[-2], st.shape[-1])[:, burn_in:, :].reshape(-1, 2)
    M = st[:, 0].astype(np.float64)
    B = st[:, 1].astype(np.float64)
    E = -float(J) * B - float(h) * M
    out = {}
    out[("E", "J")] = fluctuation_grad(E / N, -B / N, -B, beta)
    out[("E", "h")] = fluctuation_grad(E / N, -M / N, -M, beta)
    out[("M", "J")] = fluctuation_grad(M / N, None, -B, beta)
    out[("M", "h")] = fluctuation_grad(M / N, None, -M, beta)
    return out


def nnn_grad(stats, beta, J, J2, h, N, burn_in=0):
    """First and second neighbours (H = -J B - J2 B2 - h M): stats [..., T, 3]
    integer (M, B, B2) per sweep; dH/dJ2 = -B2 and, for O = E/N, dO/dJ2 = -B2/N.

    Returns {(O, theta)} for O in ('E', 'M') and theta in ('J', 'h', 'J2')."""
    st = np.asarray(stats)
    st = st.reshape(-1, st.shape[-2], st.shape[-1])[:, burn_in:, :].reshape(-1, 3)
    M, B, B2 = (st[:, k].astype(np.float64) for k in range(3))
    E = -float(J) * B - float(J2) * B2 - float(h) * M
    out = {}
    for name, X in (("J", B), ("h", M), ("J2", B2)):
        out[("E", name)] = fluctuation_grad(E / N, -X / N, -X, beta)
        out[("M", name)] = fluctuation_grad(M / N, None, -X, beta)
    return out


def cpm_pairs(n_types):
    return [(a, b) for a in range(n_types) for b in range(a, n_types)]


def cpm_grad(stats, Jtab, lam, T, N, burn_in=0):
    """stats: [..., T, n_pairs + 2] = (C_ab for a<=b, V2, V1) per Monte Carlo step.

    Returns a dict: ('J', a, b) -> d<O>/dJ_ab, 'lambda' and 'A' -> derivatives
    of O = adhesion energy per site.
    """
    Jtab = np.asarray(Jtab, dtype=np.float64)
    n_types = Jtab.shape[0]
    pairs = cpm_pairs(n_types)
    st = np.asarray(stats)
    st = st.reshape(-1, st.shape[-2], st.shape[-1])[:, burn_in:, :].reshape(-1, st.shape[-1])
    C = st[:, :len(pairs)].astype(np.float64)
    V2 = st[:, len(pairs)].astype(np.float64)
    V1 = st[:, len(pairs) + 1].astype(np.float64)
    Ead = sum(Jtab[a, b] * C[:, i] for i, (a, b) in enumerate(pairs))
    O = Ead / N
    beta = 1.0 / float(T)
    out = {}
    for i, (a, b) in enumerate(pairs):
        out[("J", a, b)] = fluctuation_grad(O, C[:, i] / N, C[:, i], beta)
    out["lambda"] = fluctuation_grad(O, None, V2, beta)
    out["A"] = fluctuation_grad(O, None, -2.0 * float(lam) * V1, beta)
    return out

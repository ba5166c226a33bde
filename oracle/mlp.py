"""Float64 reference of the 3 -> 64 -> 64 -> 2 surrogate MLP -- TEST INFRASTRUCTURE ONLY.

The paper has no surrogate; the network maps (beta, J, h) to the chain's
(<E>/N, <M>/N) and warm-starts the parameter fit.  Layers: affine input
normalisation x' = (x - mu) * inv_sigma, then Linear(3, 64) + ReLU,
Linear(64, 64) + ReLU, Linear(64, 2).  Loss: L = (1 / (2 n)) sum_i |y_i - t_i|^2.

Everything is float64 numpy; matrix products use numpy's matmul as the only
library primitive.  Adam follows Kingma & Ba (2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

LAYERS = (3, 64, 64, 2)
PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes():
    d0, d1, d2, d3 = LAYERS
    return {"W1": (d1, d0), "b1": (d1,), "W2": (d2, d1), "b2": (d2,), "W3": (d3, d2), "b3": (d3,)}


def forward(p, X, mu, inv_sigma):
    """Returns (Y, cache).  X: [n, 3]."""
    X = np.asarray(X, dtype=np.float64)
    xn = (X - np.asarray(mu, dtype=np.float64)) * np.asarray(inv_sigma, dtype=np.float64)
    z1 = xn @ p["W1"].T + p["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = np.maximum(z2, 0.0)
    Y = a2 @ p["W3"].T + p["b3"]
    return Y, (xn, z1, a1, z2, a2)


def loss(Y, T):
    d = np.asarray(Y, dtype=np.float64) - np.asarray(T, dtype=np.float64)
    return 0.5 * float(np.sum(d * d)) / d.shape[0]


def backward(p, cache, Y, T, inv_sigma, dY=None):
    """Gradients of the loss (or of sum(Y * dY) if dY is given) w.r.t. the
    parameters and the raw inputs X."""
    xn, z1, a1, z2, a2 = cache
    if dY is None:
        dY = (np.asarray(Y) - np.asarray(T)) / Y.shape[0]
    g = {}
    g["W3"] = dY.T @ a2
    g["b3"] = dY.sum(axis=0)
    da2 = dY @ p["W3"]
    dz2 = da2 * (z2 > 0.0)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(axis=0)
    da1 = dz2 @ p["W2"]
    dz1 = da1 * (z1 > 0.0)
    g["W1"] = dz1.T @ xn
    g["b1"] = dz1.sum(axis=0)
    dxn = dz1 @ p["W1"]
    dX = dxn * np.asarray(inv_sigma, dtype=np.float64)
    return g, dX


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; step counts from 1."""
    for k in PARAM_NAMES:
        m[k] = b1 * m[k] + (1.0 - b1) * g[k]
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k]
        mh = m[k] / (1.0 - b1 ** step)
        vh = v[k] / (1.0 - b2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)

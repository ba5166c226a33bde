"""Per-element error scales for the BF16 surrogate MLP kernels against the
float64 oracle.

The kernels round the weights, the normalised input, both hidden
activations and the backward signal dz2 (before the tensor-core products
dz2 W2 and dz2^T h1 and the bias gradient sum) to BF16 (8 significant bits:
one rounding changes a value by at most u = 2^-8 of its magnitude) and
accumulate in FP32 (unit roundoff 2^-24).  The oracle runs in float64 with the same BF16 weights, so the two
differ only by these roundings and their propagation through the network.

Worst-case (Wilkinson) bounds add the magnitudes of all rounding errors; in a
layer of 64 random-signed weights they overstate the error by about the
square root of the layer width per layer, far too loose to catch one wrong
gradient entry.  `scales` instead follows probabilistic rounding-error
analysis (Higham & Mary, SIAM J. Sci. Comput. 41 (2019) A2815): rounding
errors are independent and zero-mean, so a sum's error scale is the
root-sum-square of its terms' error scales.  Each intermediate value gets
such a scale, propagated from the oracle's own values and weights:

    forward   xn = bf(x') | z1 = W1 xn + b1 | h1 = bf(relu z1) | z2, a2 likewise | Y
    backward  dy = (Y - T) / n | dz2 = bf((W3^T dy) [z2 > 0]) | dz1 = (W2^T dz2) [z1 > 0]
              gradients = sums over samples of products | dX = (W1^T dz1) inv

A ReLU mask may differ between the two sides only where |z| is within K
error scales of zero; there the scale of the masked value is the whole
unmasked value plus its own scale.  The caller compares every element of the
kernels' output with the oracle's and allows K scales (K = 8: the chance
that a zero-mean error exceeds eight standard deviations is negligible).
"""
from __future__ import annotations

import numpy as np

U_BF16 = 2.0 ** -8
E_FP32 = 2.0 ** -24
K_DEFAULT = 8.0


def _rss(*terms):
    return np.sqrt(sum(t * t for t in terms))


def _mv(err, W):
    """Error scale of err @ W (independent errors: sqrt((err^2) @ W^2))."""
    return np.sqrt((err * err) @ (W * W))


def scales(p, X, mu, inv, T, K=K_DEFAULT):
    """p: oracle parameters (BF16-rounded weights, float64); X, T: [n, 3], [n, 2].

    Returns (values, scales): dicts of the oracle's Y, the six gradients and
    dX, and of their error scales (same shapes)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    inv = np.asarray(inv, dtype=np.float64)
    n = X.shape[0]
    W1, W2, W3 = p["W1"], p["W2"], p["W3"]
    acc = lambda mag, m: np.sqrt(m) * E_FP32 * mag     # FP32 accumulation of m terms
    # forward
    xn = (X - mu) * inv
    s_xn = U_BF16 * np.abs(xn)
    z1 = xn @ W1.T + p["b1"]
    s_z1 = _rss(_mv(s_xn, W1.T), acc(np.abs(xn) @ np.abs(W1.T) + np.abs(p["b1"]), 4))
    h1 = np.maximum(z1, 0.0)
    s_h1 = _rss(s_z1, U_BF16 * h1)
    z2 = h1 @ W2.T + p["b2"]
    s_z2 = _rss(_mv(s_h1, W2.T), acc(h1 @ np.abs(W2.T) + np.abs(p["b2"]), 65))
    a2 = np.maximum(z2, 0.0)
    s_a2 = _rss(s_z2, U_BF16 * a2)
    Y = a2 @ W3.T + p["b3"]
    s_Y = _rss(_mv(s_a2, W3.T), acc(a2 @ np.abs(W3.T) + np.abs(p["b3"]), 65))
    # backward
    dy = (Y - T) / n
    s_dy = _rss(s_Y / n, 2 * E_FP32 * np.abs(dy))
    da2 = dy @ W3
    s_da2 = _rss(_mv(s_dy, W3), acc(np.abs(dy) @ np.abs(W3), 2))
    dz2 = da2 * (z2 > 0.0)
    s_dz2 = np.where(np.abs(z2) <= K * s_z2, np.abs(da2) + s_da2, s_da2 * (z2 > 0.0))
    s_dz2 = _rss(s_dz2, U_BF16 * np.abs(dz2))       # the BF16 rounding of dz2
    da1 = dz2 @ W2
    s_da1 = _rss(_mv(s_dz2, W2), acc(np.abs(dz2) @ np.abs(W2), 64))
    dz1 = da1 * (z1 > 0.0)
    s_dz1 = np.where(np.abs(z1) <= K * s_z1, np.abs(da1) + s_da1, s_da1 * (z1 > 0.0))
    dxn = dz1 @ W1
    s_dX = _rss(_mv(s_dz1, W1), acc(np.abs(dz1) @ np.abs(W1), 64)) * np.abs(inv)
    # sums over samples of products a_s b_s: error scale rss_s(s_a |b| + |a| s_b)
    def outer(a, sa, b, sb):
        return np.sqrt((sa * sa).T @ (b * b) + (a * a).T @ (sb * sb)) + acc(np.abs(a).T @ np.abs(b), n)

    def colsum(a, sa):
        return np.sqrt((sa * sa).sum(0)) + acc(np.abs(a).sum(0), n)

    vals = {"Y": Y, "dX": dxn * inv,
            "W1": dz1.T @ xn, "b1": dz1.sum(0), "W2": dz2.T @ h1, "b2": dz2.sum(0),
            "W3": dy.T @ a2, "b3": dy.sum(0)}
    sc = {"Y": s_Y, "dX": s_dX,
          "W1": outer(dz1, s_dz1, xn, s_xn), "b1": colsum(dz1, s_dz1),
          "W2": outer(dz2, s_dz2, h1, s_h1), "b2": colsum(dz2, s_dz2),
          "W3": outer(dy, s_dy, a2, s_a2), "b3": colsum(dy, s_dy)}
    return vals, sc


def violations(got, vals, sc, K=K_DEFAULT, floor=1e-30):
    """{name: number of elements with |got - oracle| > K * scale + floor}."""
    bad = {}
    for k, v in vals.items():
        g = np.asarray(got[k], dtype=np.float64).reshape(v.shape)
        over = np.abs(g - v) > K * sc[k] + floor
        if over.any():
            bad[k] = int(over.sum())
    return bad


def worst_ratio(got, vals, sc, floor=1e-30):
    """max over elements of |got - oracle| / (scale + floor), per name."""
    return {k: float(np.max(np.abs(np.asarray(got[k], dtype=np.float64).reshape(v.shape) - v)
                            / (sc[k] + floor))) for k, v in vals.items()}


def emulate_fp32(p, X, mu, inv, T):
    """The kernels' arithmetic in plain torch float32 on the CPU (BF16 weights
    p, BF16 rounding of the normalised input, of both hidden activations and
    of dz2), with torch's own summation order: {Y, W1, b1, W2, b2, W3, b3, dX}."""
    import torch
    bf = lambda t: t.to(torch.bfloat16).float()
    P = {k: torch.as_tensor(np.asarray(v)).float() for k, v in p.items()}
    X, T = torch.as_tensor(np.asarray(X)).float(), torch.as_tensor(np.asarray(T)).float()
    mu, inv = torch.as_tensor(np.asarray(mu)).float(), torch.as_tensor(np.asarray(inv)).float()
    xn = bf((X - mu) * inv)
    h1 = bf(torch.relu(xn @ P["W1"].T + P["b1"]))
    a2 = bf(torch.relu(h1 @ P["W2"].T + P["b2"]))
    Y = a2 @ P["W3"].T + P["b3"]
    dy = (Y - T) / X.shape[0]
    dz2 = bf((dy @ P["W3"]) * (a2 > 0))
    dz1 = (dz2 @ P["W2"]) * (h1 > 0)
    out = {"Y": Y, "W1": dz1.T @ xn, "b1": dz1.sum(0), "W2": dz2.T @ h1, "b2": dz2.sum(0),
           "W3": dy.T @ a2, "b3": dy.sum(0), "dX": (dz1 @ P["W1"]) * inv}
    return {k: v.double().numpy() for k, v in out.items()}

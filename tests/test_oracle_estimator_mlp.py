"""Pins for the oracle's fluctuation estimator and float64 MLP (CPU only)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import estimator, mlp
from tests import exact


@pytest.mark.parametrize("beta,J,h", [(0.3, 1.0, 0.1), (0.44, 1.0, 0.0), (0.6, 0.8, -0.2)])
def test_exact_fluctuation_identity_equals_finite_differences(beta, J, h):
    """The identity d<O>/dtheta = <dO> - beta Cov(O, dH) holds exactly on the
    4x4 enumeration: compare with central differences of exact means."""
    g = exact.ising_exact_grad(beta, J, h)
    N, d = 16, 1e-5
    mean = lambda b, j, hh, key: exact.ising_exact(b, j, hh)[key] / N
    fd = {
        ("E", "J"): (mean(beta, J + d, h, "E") - mean(beta, J - d, h, "E")) / (2 * d),
        ("E", "h"): (mean(beta, J, h + d, "E") - mean(beta, J, h - d, "E")) / (2 * d),
        ("M", "J"): (mean(beta, J + d, h, "M") - mean(beta, J - d, h, "M")) / (2 * d),
        ("M", "h"): (mean(beta, J, h + d, "M") - mean(beta, J, h - d, "M")) / (2 * d),
    }
    for k in fd:
        assert abs(g[k] - fd[k]) < 1e-6 * max(1.0, abs(fd[k])), (k, g[k], fd[k])


def test_estimator_on_exact_samples_converges_to_exact_gradient():
    """Samples drawn i.i.d. from the exact law: the oracle's estimator must
    agree with the exact gradient within a few standard errors."""
    beta, J, h = 0.4, 1.0, 0.15
    ex = exact.ising_exact(beta, J, h)
    rng = np.random.default_rng(3)
    idx = rng.choice(len(ex["w"]), size=400000, p=ex["w"])
    st = np.stack([ex["Mall"][idx], ex["Ball"][idx]], axis=1).astype(np.int64)
    g = estimator.ising_grad(st[None], beta, J, h, 16)
    want = exact.ising_exact_grad(beta, J, h)
    # split into 20 batches for an error bar
    parts = [estimator.ising_grad(p[None], beta, J, h, 16) for p in np.array_split(st, 20)]
    for k in want:
        err = np.std([p[k] for p in parts], ddof=1) / np.sqrt(20)
        assert abs(g[k] - want[k]) < 5 * err + 1e-9, (k, g[k], want[k], err)


def test_estimator_on_oracle_chain_matches_exact_gradient():
    beta, J, h = 0.35, 1.0, 0.1
    chains = []
    for c in range(8):
        s = oracle.init_ising(4, 100 + c, c).copy()
        chains.append(oracle.ising_run(s, beta, J, h, 100 + c, c, 0, 30000))
    st = np.stack(chains)
    g = estimator.ising_grad(st, beta, J, h, 16, burn_in=200)
    per = [estimator.ising_grad(st[i:i + 1], beta, J, h, 16, burn_in=200) for i in range(8)]
    want = exact.ising_exact_grad(beta, J, h)
    for k in want:
        err = np.std([p[k] for p in per], ddof=1) / np.sqrt(8)
        assert abs(g[k] - want[k]) < 5 * err + 1e-9, (k, g[k], want[k], err)


def test_cpm_estimator_medium_medium_gradient_is_zero_and_shapes():
    p = oracle.CPM(L=24, J=[[0, 16, 16], [16, 2, 11], [16, 11, 14]], lam=1, target=16,
                   n_cells=9, T=8.0, side=4, cols=3)
    ids, types, vol = p.init(2)
    ids = ids.copy()
    st = p.run(ids, vol, types, 2, 0, 0, 200)
    g = estimator.cpm_grad(st, p.J, p.lam, p.T, 24 * 24, burn_in=50)
    assert g[("J", 0, 0)] == 0.0
    # explicit term: d<O>/dJ_ab contains <C_ab>/N > 0 for pairs that touch
    assert set(k for k in g if isinstance(k, tuple)) == {("J", a, b) for a in range(3) for b in range(a, 3)}


# ---------------------------------------------------------------------------
# MLP reference vs torch (float64) -- an independent library implementation
# ---------------------------------------------------------------------------
def _params(seed=0):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(0, 0.5, size=s) for k, s in mlp.shapes().items()}


def _torch_model(p):
    net = torch.nn.Sequential(torch.nn.Linear(3, 64), torch.nn.ReLU(), torch.nn.Linear(64, 64),
                              torch.nn.ReLU(), torch.nn.Linear(64, 2)).double()
    with torch.no_grad():
        for i, (w, b) in enumerate([("W1", "b1"), ("W2", "b2"), ("W3", "b3")]):
            net[2 * i].weight.copy_(torch.from_numpy(p[w]))
            net[2 * i].bias.copy_(torch.from_numpy(p[b]))
    return net


def test_mlp_forward_backward_match_torch_autograd():
    p = _params()
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(37, 3))
    T = rng.normal(size=(37, 2))
    mu, inv = np.array([0.1, -0.2, 0.3]), np.array([2.0, 0.5, 1.5])
    Y, cache = mlp.forward(p, X, mu, inv)
    g, dX = mlp.backward(p, cache, Y, T, inv)
    net = _torch_model(p)
    Xt = torch.from_numpy(X).requires_grad_(True)
    Yt = net((Xt - torch.from_numpy(mu)) * torch.from_numpy(inv))
    Lt = 0.5 * ((Yt - torch.from_numpy(T)) ** 2).sum() / X.shape[0]
    Lt.backward()
    assert np.allclose(Y, Yt.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert abs(mlp.loss(Y, T) - Lt.item()) < 1e-12
    for i, (w, b) in enumerate([("W1", "b1"), ("W2", "b2"), ("W3", "b3")]):
        assert np.allclose(g[w], net[2 * i].weight.grad.numpy(), rtol=1e-12, atol=1e-13)
        assert np.allclose(g[b], net[2 * i].bias.grad.numpy(), rtol=1e-12, atol=1e-13)
    assert np.allclose(dX, Xt.grad.numpy(), rtol=1e-12, atol=1e-13)


def test_mlp_adam_matches_torch_adam():
    p = _params(2)
    net = _torch_model(p)
    opt = torch.optim.Adam(net.parameters(), lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    rng = np.random.default_rng(5)
    mu, inv = np.zeros(3), np.ones(3)
    for step in range(1, 4):
        X = rng.uniform(-1, 1, size=(16, 3))
        T = rng.normal(size=(16, 2))
        Y, cache = mlp.forward(p, X, mu, inv)
        g, _ = mlp.backward(p, cache, Y, T, inv)
        mlp.adam_step(p, g, m, v, step, 1e-2)
        opt.zero_grad()
        Lt = 0.5 * ((net(torch.from_numpy(X)) - torch.from_numpy(T)) ** 2).sum() / 16
        Lt.backward()
        opt.step()
    for i, (w, b) in enumerate([("W1", "b1"), ("W2", "b2"), ("W3", "b3")]):
        assert np.allclose(p[w], net[2 * i].weight.detach().numpy(), rtol=1e-10, atol=1e-12)
        assert np.allclose(p[b], net[2 * i].bias.detach().numpy(), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("lam", [1, 2])
def test_cpm_estimator_area_and_lambda_entries_from_energy_differences(lam):
    """Eq. "h": H = adhesion + lambda * sum_cells (a - A)^2 (medium excluded).
    On the oracle chain's own states, dH/dlambda and dH/dA are formed as exact
    integer differences of the full energy (or_cpm_energy at lambda + 1 and at
    A +- 1) and the adhesion O as the energy at lambda = 0; the fluctuation
    formula on those per-sample values must give the estimator's 'lambda' and
    'A' entries.  A dropped factor 2 or lambda, or a sign, fails here."""
    J = [[0, 16, 16], [16, 2, 11], [16, 11, 14]]
    p = oracle.CPM(L=24, J=J, lam=lam, target=16, n_cells=9, T=6.0, side=4, cols=3)
    at = lambda **kw: oracle.CPM(L=24, J=J, lam=kw.get("lam", lam), target=kw.get("target", 16),
                                 n_cells=9, T=6.0, side=4, cols=3)
    ids, types, vol = p.init(4)
    ids = ids.copy()
    O, dlam, dA, stats = [], [], [], []
    for t in range(120):
        stats.append(p.run(ids, vol, types, 4, 0, t, 1)[0])
        if t < 20:
            continue
        H = p.energy(ids, types)
        O.append(at(lam=0).energy(ids, types))
        dlam.append(at(lam=lam + 1).energy(ids, types) - H)
        hp, hm = at(target=17).energy(ids, types), at(target=15).energy(ids, types)
        assert (hp - hm) % 2 == 0
        dA.append((hp - hm) // 2)
    st = np.array(stats)[20:]
    V2, V1 = st[:, -2], st[:, -1]
    assert np.array_equal(dlam, V2)                    # dH/dlambda = sum (a - A)^2
    assert np.array_equal(dA, -2 * lam * V1)           # dH/dA = -2 lambda sum (a - A)
    pairs = estimator.cpm_pairs(3)
    Ead = sum(J[a][b] * st[:, i] for i, (a, b) in enumerate(pairs))
    assert np.array_equal(O, Ead)                      # adhesion energy from the contacts
    O = np.asarray(O, dtype=np.float64) / (24 * 24)
    g = estimator.cpm_grad(st[None], J, lam, p.T, 24 * 24)
    beta = 1.0 / p.T
    for key, dH in (("lambda", dlam), ("A", dA)):
        dH = np.asarray(dH, dtype=np.float64)
        want = -beta * float(np.mean((O - O.mean()) * (dH - dH.mean())))
        assert abs(g[key] - want) <= 1e-12 * max(1.0, abs(want)), (key, g[key], want)
    assert g["A"] != 0.0 and g["lambda"] != 0.0


# ---------------------------------------------------------------------------
# Per-element error scales of the BF16 kernels (tests/mlp_bounds.py)
# ---------------------------------------------------------------------------
def _bf16_params(seed, scale):
    rng = np.random.default_rng(seed)
    return {k: torch.from_numpy(rng.normal(0, scale, size=s)).to(torch.bfloat16).double().numpy()
            for k, s in mlp.shapes().items()}


@pytest.mark.parametrize("seed,scale,n", [(0, 0.3, 333), (1, 0.5, 1000), (2, 0.15, 128)])
def test_mlp_error_scales_cover_the_kernel_arithmetic_and_catch_planted_mistakes(seed, scale, n):
    """The kernels' arithmetic emulated in float32 (BF16 roundings at the same
    places) stays within K error scales of the float64 oracle, element by
    element; mistakes planted in the oracle's outputs are flagged."""
    from tests import mlp_bounds as mb
    p = _bf16_params(seed, scale)
    rng = np.random.default_rng(100 + seed)
    X = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    T = (0.5 * rng.normal(size=(n, 2))).astype(np.float32)
    mu = np.array([0.1, -0.2, 0.05], dtype=np.float32)
    inv = np.array([2.0, 1.5, 3.0], dtype=np.float32)
    vals, sc = mb.scales(p, X, mu, inv, T)
    # the scales' values are the oracle's own forward and backward
    Y, cache = mlp.forward(p, X, mu, inv)
    g, dX = mlp.backward(p, cache, Y, T, inv)
    assert np.allclose(vals["Y"], Y, rtol=1e-13, atol=1e-15) and np.allclose(vals["dX"], dX, rtol=1e-12, atol=1e-15)
    for k in g:
        assert np.allclose(vals[k], g[k], rtol=1e-12, atol=1e-15), k
    em = mb.emulate_fp32(p, X, mu, inv, T)
    assert mb.violations(em, vals, sc) == {}, mb.worst_ratio(em, vals, sc)
    # planted: one W2 gradient entry 25% off, the W2 gradient transposed,
    # the layer-1 ReLU mask dropped in the backward pass, b3's sign flipped
    k = np.unravel_index(np.argmax(np.abs(vals["W2"])), vals["W2"].shape)
    wrong = dict(vals, W2=vals["W2"].copy())
    wrong["W2"][k] *= 1.25
    assert mb.violations(wrong, vals, sc).get("W2") == 1
    assert mb.violations(dict(vals, W2=vals["W2"].T.copy()), vals, sc).get("W2", 0) > 100
    xn, z1, a1, z2, a2 = cache
    dz2 = ((Y - T) / n @ p["W3"]) * (z2 > 0)
    nomask = (dz2 @ p["W2"]).T @ xn
    assert mb.violations(dict(vals, W1=nomask), vals, sc).get("W1", 0) > 10
    assert mb.violations(dict(vals, b3=-vals["b3"]), vals, sc).get("b3") == 2

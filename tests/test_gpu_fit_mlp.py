"""GPU checks of the gradient path and the BF16 surrogate.

* MLP forward / backward kernels against the float64 oracle, element by
  element: the kernels round the normalised input and both hidden
  activations to BF16 (8 significant bits) and accumulate in FP32; every
  element must lie within K error scales propagated from those roundings
  (tests/mlp_bounds.py).
* The Adam kernel against the oracle's Adam (float32 vs float64).
* The fluctuation-estimator gradient against exact 4x4 enumeration and
  against finite differences of Monte Carlo means.
* The (J, h) fit driven by the estimator, with and without the surrogate
  warm start (the warm start reaches the tolerance in fewer steps).
"""
import numpy as np
import pytest
import torch

import paper_2304_01772_gb300 as sm
from oracle import mlp as omlp
from paper_2304_01772_gb300 import fit
from tests import exact

pytestmark = pytest.mark.gpu


def _oracle_params(flat):
    p = flat.detach().to(torch.bfloat16).double().cpu().numpy()
    out, off = {}, 0
    for k, shp in omlp.shapes().items():
        n = int(np.prod(shp))
        out[k] = p[off:off + n].reshape(shp)
        off += n
    return out


def _flat(d):
    return np.concatenate([d[k].ravel() for k in omlp.PARAM_NAMES])


def test_mlp_kernels_match_oracle():
    """Every output element, gradient entry and input gradient of the kernels
    lies within K = 8 error scales of the float64 oracle's (BF16 roundings
    of the normalised input and both hidden activations, FP32 accumulation;
    the scales and their calibration are in tests/mlp_bounds.py)."""
    from tests import mlp_bounds as mb
    s = fit.Surrogate(seed=11)
    g = torch.Generator().manual_seed(0)
    s.params += 0.05 * torch.randn(s.params.shape, generator=g).cuda()   # non-zero biases too
    X = torch.from_numpy(fit.sample_box(333, seed=5)).cuda()                # 333: ragged last block
    T = (0.5 * torch.randn((333, 2), generator=g)).cuda()
    Y = sm.mlp_forward(s.params, s.mu, s.inv_sigma, X)
    grad, loss, dX = sm.mlp_backward(s.params, s.mu, s.inv_sigma, X, T, want_dx=True)
    p = _oracle_params(s.params)
    mu, inv = s.mu.cpu().numpy(), s.inv_sigma.cpu().numpy()
    Xh, Th = X.cpu().numpy(), T.cpu().numpy()
    vals, sc = mb.scales(p, Xh, mu, inv, Th)
    gflat = grad.cpu().numpy().astype(np.float64)
    got, off = {"Y": Y.cpu().numpy(), "dX": dX.cpu().numpy()}, 0
    for k, shp in omlp.shapes().items():
        n = int(np.prod(shp))
        got[k] = gflat[off:off + n].reshape(shp)
        off += n
    assert mb.violations(got, vals, sc) == {}, mb.worst_ratio(got, vals, sc)
    # the loss: one FP32 sum of n squared errors, each off by its Y scale
    Lo = omlp.loss(vals["Y"], Th)
    s_loss = np.sqrt(np.sum((np.abs(vals["Y"] - Th) * sc["Y"]) ** 2)) / 333 + 333 * 2.0 ** -24 * Lo
    assert abs(float(loss) - Lo) <= mb.K_DEFAULT * s_loss, (float(loss), Lo, s_loss)
    # the same arithmetic emulated in float32 on the CPU agrees as closely
    em = mb.emulate_fp32(p, Xh, mu, inv, Th)
    assert mb.violations(em, vals, sc) == {}


def test_adam_kernel_matches_oracle():
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=sm.mlp_param_count()).astype(np.float32)
    params = torch.from_numpy(p0.copy()).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    shapes = omlp.shapes()
    po = {}
    off = 0
    for k in omlp.PARAM_NAMES:
        n = int(np.prod(shapes[k]))
        po[k] = p0[off:off + n].astype(np.float64).reshape(shapes[k])
        off += n
    mo = {k: np.zeros_like(x) for k, x in po.items()}
    vo = {k: np.zeros_like(x) for k, x in po.items()}
    for step in range(1, 4):
        gflat = rng.normal(size=p0.size).astype(np.float32)
        sm.adam(params, torch.from_numpy(gflat).cuda(), m, v, step, 1e-2)
        go, off = {}, 0
        for k in omlp.PARAM_NAMES:
            n = int(np.prod(shapes[k]))
            go[k] = gflat[off:off + n].astype(np.float64).reshape(shapes[k])
            off += n
        omlp.adam_step(po, go, mo, vo, step, 1e-2)
    np.testing.assert_allclose(params.cpu().numpy(), _flat(po), rtol=1e-5, atol=1e-6)


def test_estimator_matches_exact_4x4_gradients():
    beta, J, h = 0.35, 1.0, 0.1
    want = exact.ising_exact_grad(beta, J, h)
    ex = exact.ising_exact(beta, J, h)
    ests, means = [], []
    for rep in range(8):
        sim = sm.Sim(sm.SPIN_ISING, [dict(L=4, beta=beta, J=J, h=h)] * 512, seed=100 + rep, max_record=400)
        sim.sweep(200)
        sim.sweep(400, record=True)
        gE = sim.grad(0, 400, observable=0, pool=True).cpu().numpy()[0]
        gM = sim.grad(0, 400, observable=1, pool=True).cpu().numpy()[0]
        ests.append([gE[0], gE[1], gM[0], gM[1]])
        means.append(sim.expectations(0, 400, pool=True).cpu().numpy()[0])
        sim.close()
    ests = np.array(ests)
    means = np.array(means)
    keys = [("E", "J"), ("E", "h"), ("M", "J"), ("M", "h")]
    for i, k in enumerate(keys):
        err = ests[:, i].std(ddof=1) / np.sqrt(len(ests))
        assert abs(ests[:, i].mean() - want[k]) < 5 * err + 1e-4, (k, ests[:, i].mean(), want[k], err)
    for i, (name, val) in enumerate([("E", ex["E"] / 16), ("M", ex["M"] / 16)]):
        err = means[:, i].std(ddof=1) / np.sqrt(len(means))
        assert abs(means[:, i].mean() - val) < 5 * err + 1e-4, (name, means[:, i].mean(), val)


def test_estimator_matches_finite_differences():
    """d<E>/N/dJ and d<M>/N/dh from the estimator vs central differences of
    Monte Carlo means with common random numbers."""
    beta, J, h, d = 0.4, 0.9, 0.05, 0.02

    def run(JJ, hh):
        sim = sm.Sim(sm.SPIN_ISING, [dict(L=32, beta=beta, J=JJ, h=hh)] * 64, seed=5, max_record=600)
        sim.sweep(300)
        sim.sweep(600, record=True)
        e = sim.expectations(0, 600, pool=True).cpu().numpy()[0]
        g = (sim.grad(0, 600, observable=0, pool=True).cpu().numpy()[0],
             sim.grad(0, 600, observable=1, pool=True).cpu().numpy()[0])
        sim.close()
        return e, g

    e0, (gE, gM) = run(J, h)
    fdEJ = (run(J + d, h)[0][0] - run(J - d, h)[0][0]) / (2 * d)
    fdMh = (run(J, h + d)[0][1] - run(J, h - d)[0][1]) / (2 * d)
    assert abs(gE[0] - fdEJ) < 0.2 * abs(fdEJ), (gE[0], fdEJ)
    assert abs(gM[1] - fdMh) < 0.25 * abs(fdMh), (gM[1], fdMh)


def test_fit_reaches_target_and_surrogate_warm_start_helps():
    target, beta = (-1.2, 0.5), 0.45
    # surrogate: 2048 chains of 32^2 in one batched run, then training
    X = torch.from_numpy(fit.sample_box(2048, seed=1)).cuda()
    Y = fit.chain_targets(X, L=32, n_burn=300, n_meas=300)
    sur = fit.Surrogate(seed=3)
    losses = sur.train(X, Y, epochs=1500, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    rms = float(((sur.predict(X) - Y) ** 2).mean().sqrt())
    theta_w = sur.invert(target, beta).cpu().numpy()
    assert 0.5 <= theta_w[0] <= 1.5 and -0.2 <= theta_w[1] <= 0.2

    def run_fit(theta0, max_steps):
        ens = fit.IsingEnsemble(32, 64, beta, seed=21, n_burn=150, n_meas=150)
        hist = []
        th, steps, loss = fit.fit(ens, target, theta0, lr=1e-2, max_steps=max_steps, tol=2e-3, history=hist)
        return steps, loss, hist

    cold_steps, cold_loss, cold_hist = run_fit((1.0, 0.0), 60)
    warm_steps, warm_loss, _ = run_fit(tuple(float(x) for x in theta_w), 60)
    print(f"surrogate rms {rms:.4f}; warm start {theta_w}; steps to loss < 2e-3: cold {cold_steps} "
          f"(loss {cold_hist[0][-1]:.3f} -> {cold_loss:.4f}), warm {warm_steps} (loss {warm_loss:.5f})")
    # the Monte Carlo gradient drives the fit: the loss falls by an order of magnitude
    assert cold_loss < 0.1 * cold_hist[0][-1]
    # the surrogate's warm start reaches the tolerance, in fewer gradient steps
    assert warm_loss < 2e-3
    assert warm_steps < cold_steps


def test_pooled_gradient_over_two_contexts_via_limbs():
    """The multi-GPU exchange emulated with two contexts (two ranks' chains
    sharing theta): their limbs summed element-wise give the estimator over
    both sample sets, as the float64 oracle computes it from the records."""
    from oracle import estimator
    beta, J, h, L, n = 0.42, 1.0, 0.03, 32, 300
    sims = [sm.Sim(sm.SPIN_ISING, [dict(L=L, beta=beta, J=J, h=h)] * 16, seed=s, max_record=n) for s in (11, 12)]
    recs = []
    for x in sims:
        x.sweep(50)
        x.sweep(n, record=True)
        recs.append(x.observables_host(0, n)[0])          # [n, lattices, 2]
    limbs = sims[0].pooled_limbs(0, n) + sims[1].pooled_limbs(0, n)
    g, e = sims[0].grad_from_limbs(limbs, observable=0)
    gm, _ = sims[0].grad_from_limbs(limbs, observable=1)
    st = np.concatenate([r.transpose(1, 0, 2) for r in recs], axis=0)   # [chains, n, 2]
    ref = estimator.ising_grad(st, np.float32(beta), np.float32(J), np.float32(h), L * L)
    np.testing.assert_allclose(g.cpu().numpy()[0], [ref[("E", "J")], ref[("E", "h")]], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(gm.cpu().numpy()[0], [ref[("M", "J")], ref[("M", "h")]], rtol=1e-9, atol=1e-12)
    Ms = st[..., 0].astype(np.float64) / (L * L)
    Es = (-float(np.float32(J)) * st[..., 1] - float(np.float32(h)) * st[..., 0]) / (L * L)
    np.testing.assert_allclose(e.cpu().numpy()[0], [Es.mean(), Ms.mean()], rtol=1e-12)
    # one context's limbs alone reproduce its own pooled gradient exactly
    g0, _ = sims[0].grad_from_limbs(sims[0].pooled_limbs(0, n), observable=0)
    assert torch.equal(g0, sims[0].grad(0, n, observable=0, pool=True))


def test_observables_fn_backward_is_the_estimator_jacobian():
    """The torch.autograd.Function around the ensemble: forward returns the
    pooled expectations of the recorded samples, backward returns the upstream
    gradient times the pooled fluctuation-estimator Jacobian of the same samples
    (checked against spin_grad on a second ensemble with the same seed)."""
    ens = fit.IsingEnsemble(8, 32, 0.44, seed=11, n_burn=50, n_meas=100, tune=False)
    theta = torch.tensor([0.9, 0.05], dtype=torch.float64, device="cuda", requires_grad=True)
    out = fit.ObservablesFn.apply(theta, ens)
    w = torch.tensor([0.7, -1.3], dtype=torch.float64, device="cuda")
    (out * w).sum().backward()
    ref = sm.Sim(sm.SPIN_ISING, [dict(L=32, beta=0.44, J=0.9, h=0.05)] * 8, seed=11, max_record=100)
    ref.sweep(50)
    ref.sweep(100, record=True)
    e = ref.expectations(0, 100, pool=True)[0]
    jac = torch.stack([ref.grad(0, 100, observable=0, pool=True)[0], ref.grad(0, 100, observable=1, pool=True)[0]])
    assert torch.allclose(out.detach(), e, rtol=1e-12, atol=0)
    assert torch.allclose(theta.grad, w @ jac, rtol=1e-12, atol=1e-15)

"""Differentiable Monte Carlo fit of (J, h) and its BF16 MLP warm start.

The paper differentiates through relaxed Monte Carlo steps (Alg. 2) to tune
exchange parameters.  Here the gradient of a Monte Carlo expectation comes
from the fluctuation estimator computed by the library (spin_grad):

    d<O>/dtheta = <dO/dtheta> - beta (<O dH/dtheta> - <O><dH/dtheta>),

wrapped in a torch.autograd.Function so that any torch loss of (<E>/N, <M>/N)
back-propagates to (J, h).  Parameter updates use the library's Adam kernel.

The surrogate is the library's BF16 MLP 3 -> 64 -> 64 -> 2 mapping
(beta, J, h) to (<E>/N, <M>/N): trained on chain outputs produced by one
batched sweep launch over many small lattices, then inverted by gradient
descent on its inputs to pick a starting point for the Monte Carlo fit.
Every numerical step (sweeps, moments, expectations, gradients, MLP forward
and backward, Adam) runs in the library's CUDA kernels; this module only
sequences the calls.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import SPIN_ISING, Sim, adam, mlp_backward, mlp_forward, mlp_param_count
from . import workloads as wl


class IsingEnsemble:
    """n_chains Ising chains of side L sharing (beta, J, h).

    run(J, h) sets the parameters, runs n_burn + n_meas sweeps (recording the
    last n_meas) and returns the pooled expectations [2] and the pooled
    Jacobian [2 observables][2 parameters] (d<E>/N, d<M>/N by dJ, dh), both
    float64 on the device.
    """

    def __init__(self, n_chains, L, beta, J=1.0, h=0.0, seed=0, n_burn=200, n_meas=200, tune=True):
        self.lats = [dict(L=L, beta=beta, J=J, h=h) for _ in range(n_chains)]
        self.beta = beta
        self.n_burn, self.n_meas = n_burn, n_meas
        self.sim = Sim(SPIN_ISING, self.lats, seed=seed, max_record=n_meas)
        if tune:
            # pick the fastest launch form on this batch (a few trial sweeps; the chain
            # advances, but the draws depend only on the sweep index, so results do not
            # depend on the form chosen)
            self.sim.autotune(4)
        self.sweeps = 0

    def run(self, J, h):
        for d in self.lats:
            d["J"], d["h"] = float(J), float(h)
        self.sim.set_params(self.lats)
        self.sim.sweep(self.n_burn)
        self.sim.sweep(self.n_meas, record=True)
        self.sweeps += self.n_burn + self.n_meas
        first = self.sim.n_records - self.n_meas
        exp = self.sim.expectations(first, self.n_meas, pool=True)[0]
        jac = torch.stack([self.sim.grad(first, self.n_meas, observable=0, pool=True)[0],
                           self.sim.grad(first, self.n_meas, observable=1, pool=True)[0]])
        return exp, jac


class ObservablesFn(torch.autograd.Function):
    """theta = (J, h) -> (<E>/N, <M>/N) of an IsingEnsemble; backward uses the
    fluctuation-estimator Jacobian of the same samples."""

    @staticmethod
    def forward(ctx, theta, ensemble):
        J, h = (float(x) for x in theta.detach().cpu())
        exp, jac = ensemble.run(J, h)
        ctx.save_for_backward(jac)
        return exp.to(theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (jac,) = ctx.saved_tensors
        return (grad_out.to(jac.dtype) @ jac).to(grad_out.dtype), None


def fit(ensemble, target, theta0, lr=1e-2, max_steps=200, tol=1e-3, history=None, b1=0.9, b2=0.999):
    """Adam on (J, h) until the squared error to `target` falls below tol.

    Returns (theta, steps, loss); `history` (a list) receives
    (step, J, h, E, M, loss) per step.
    """
    theta = torch.tensor(theta0, dtype=torch.float32, device="cuda")
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    tgt = torch.tensor(target, dtype=torch.float64, device="cuda")
    loss_v = math.inf
    for step in range(1, max_steps + 1):
        th = theta.double().requires_grad_(True)
        out = ObservablesFn.apply(th, ensemble)
        loss = ((out - tgt) ** 2).sum()
        loss.backward()
        loss_v = float(loss.detach())
        if history is not None:
            o = out.detach().cpu().numpy()
            history.append((step, float(theta[0]), float(theta[1]), float(o[0]), float(o[1]), loss_v))
        if loss_v < tol:
            return theta, step, loss_v
        adam(theta, th.grad.float().contiguous(), m, v, step, lr, b1, b2)
    return theta, max_steps, loss_v


# --------------------------------------------------------------------------
# surrogate
# --------------------------------------------------------------------------
BOX = ((0.3, 0.6), (0.5, 1.5), (-0.2, 0.2))   # beta, J, h


def sample_box(n, seed=1):
    r = wl.SplitMix64(seed)
    X = np.empty((n, 3), dtype=np.float32)
    for i in range(n):
        for k, (lo, hi) in enumerate(BOX):
            X[i, k] = lo + (hi - lo) * r.uniform()
    return X


def chain_targets(X, L=32, n_burn=300, n_meas=300, seed=7):
    """(<E>/N, <M>/N) of one chain per row of X from one batched launch per sweep."""
    lats = [dict(L=L, beta=float(b), J=float(j), h=float(h)) for b, j, h in X]
    sim = Sim(SPIN_ISING, lats, seed=seed, max_record=n_meas)
    sim.sweep(n_burn)
    sim.sweep(n_meas, record=True)
    Y = sim.expectations(0, n_meas).float().contiguous()
    sim.close()
    return Y


def xavier_params(seed=3):
    """Glorot-uniform weights, zero biases, flattened in the library's layout."""
    r = wl.SplitMix64(seed)
    out = []
    for fan_in, fan_out in ((3, 64), (64, 64), (64, 2)):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        out.append(np.array([(2 * r.uniform() - 1) * a for _ in range(fan_in * fan_out)], dtype=np.float32))
        out.append(np.zeros(fan_out, dtype=np.float32))
    p = np.concatenate(out)
    assert p.size == mlp_param_count()
    return torch.from_numpy(p).cuda()


class Surrogate:
    def __init__(self, seed=3):
        self.params = xavier_params(seed)
        self.mu = torch.tensor([0.5 * (lo + hi) for lo, hi in BOX], dtype=torch.float32, device="cuda")
        self.inv_sigma = torch.tensor([2.0 / (hi - lo) for lo, hi in BOX], dtype=torch.float32, device="cuda")
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0

    def predict(self, X):
        return mlp_forward(self.params, self.mu, self.inv_sigma, X)

    def train(self, X, Y, epochs=2000, lr=3e-3):
        """Full-batch Adam on the squared error; returns the loss history."""
        losses = []
        for _ in range(epochs):
            grad, loss, _ = mlp_backward(self.params, self.mu, self.inv_sigma, X, Y)
            self.step += 1
            adam(self.params, grad, self.m, self.v, self.step, lr)
            losses.append(loss)
        return torch.cat(losses).cpu().numpy()

    def invert(self, target, beta, theta0=(1.0, 0.0), steps=400, lr=1e-2):
        """Gradient descent on (J, h) through the frozen network (input gradient)."""
        th = torch.tensor(theta0, dtype=torch.float32, device="cuda")
        m = torch.zeros_like(th)
        v = torch.zeros_like(th)
        T = torch.tensor([list(target)], dtype=torch.float32, device="cuda")
        for k in range(1, steps + 1):
            X = torch.cat([torch.tensor([beta], dtype=torch.float32, device="cuda"), th]).view(1, 3).contiguous()
            _, _, dX = mlp_backward(self.params, self.mu, self.inv_sigma, X, T, want_dx=True)
            adam(th, dX[0, 1:].contiguous(), m, v, k, lr)
        return th

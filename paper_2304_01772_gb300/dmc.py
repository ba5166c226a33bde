"""Differentiable Monte Carlo (Alg. 2): pattern optimisation of the exchange
parameters (Sec. "Optimization of the exchange parameters") and energy
minimisation over the spin values (Sec. "Optimization of the spin values").

A batch of Ising lattices with one exchange parameter per bond is steered
towards target patterns: each iteration runs `sweeps` relaxed sweeps from the
current spins, takes the L2 loss to the target, back-propagates to the bond
parameters, applies Adam (lr 1e-3, beta1 0.9, beta2 0.999 as in the paper) and
discretises the spins, which carry over to the next iteration.  Every step runs
in the library's kernels (spin_dmc_*, spin_adam); this module only holds the
buffers and sequences the calls.
"""
from __future__ import annotations

import torch

from . import (adam, dmc_backward, dmc_discretize, dmc_energy, dmc_forward, dmc_loss, dmc_spin_iter,
               dmc_spin_iter_max_sweeps, dmc_spin_step, dmc_step, dmc_step_max_sweeps, dmc_tape_floats)


class PatternOptimizer:
    def __init__(self, target, beta, alpha, sweeps, seed=0, h=0.0, J0=1.0, lr=1e-3, spins=None, fused=True):
        """target: [B, L, L] float32 (+-1) on the device; spins: start state
        (default: all +1)."""
        self.target = target.contiguous()
        B, L = target.shape[0], target.shape[-1]
        self.B, self.L = B, L
        self.beta, self.alpha, self.h, self.sweeps, self.seed, self.lr = beta, alpha, h, sweeps, seed, lr
        dev = target.device
        self.J = torch.full((B, 2, L, L), float(J0), dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.J)
        self.v = torch.zeros_like(self.J)
        self.gJ = torch.zeros_like(self.J)
        self.spins = (torch.ones((B, L, L), dtype=torch.float32, device=dev) if spins is None
                      else spins.clone().contiguous())
        self.gs = torch.zeros_like(self.spins)
        self.tape = torch.empty(dmc_tape_floats(B, L, sweeps), dtype=torch.float32, device=dev)
        self.loss = torch.zeros(B, dtype=torch.float64, device=dev)
        self.step_count = 0
        self.sweep = 0
        self.fused = fused and sweeps <= dmc_step_max_sweeps(L)

    def step(self, stream=None):
        """One iteration; returns the per-lattice loss tensor (device, float64)
        of the relaxed state before the update.  A single fused launch when the
        tape fits in shared memory, else the separate calls."""
        if self.fused:
            self.step_count += 1
            dmc_step(self.seed, self.J, self.spins, self.m, self.v, self.target, self.loss, self.beta, self.h,
                     self.alpha, self.sweep, self.sweeps, self.step_count, self.lr, stream=stream)
            self.sweep += self.sweeps
            return self.loss
        return self.step_separate(stream)

    def step_separate(self, stream=None):
        """The same iteration as five launches (forward, loss, reverse pass,
        Adam, discretisation) through a tape in device memory."""
        dmc_forward(self.seed, self.J, self.spins, self.beta, self.h, self.alpha, self.sweep, self.sweeps,
                    self.tape, stream)
        dmc_loss(self.spins, self.target, self.gs, self.loss, stream)
        dmc_backward(self.seed, self.J, self.spins, self.tape, self.beta, self.h, self.alpha, self.sweep,
                     self.sweeps, self.gs, self.gJ, stream)
        self.step_count += 1
        adam(self.J, self.gJ, self.m, self.v, self.step_count, self.lr, stream=stream)
        dmc_discretize(self.spins, stream)
        self.sweep += self.sweeps
        return self.loss


def gradient_by_temperature(target, temperatures, alpha=10.0, sweeps=1, seed=0, h=0.0, J0=1.0, spins=None,
                            stream=None):
    """The temperature study of Sec. "Optimization of the exchange parameters":
    the size of the coupling gradient depends on T (at low T few spins move,
    at high T the moves hardly depend on the couplings), so there is a
    temperature where the optimisation learns fastest.  For each T (beta = 1/T)
    one iteration from the same start (couplings J0, spins all +1 unless
    given): `sweeps` relaxed sweeps, the L2 loss to the target and the reverse
    pass.  Returns [(T, mean |dL/dJ| over all bonds of all lattices, mean
    loss)]; the sweeps, loss and reverse pass run in the library's kernels."""
    out = []
    for T in temperatures:
        opt = PatternOptimizer(target, beta=1.0 / float(T), alpha=alpha, sweeps=sweeps, seed=seed, h=h, J0=J0,
                               spins=spins, fused=False)
        dmc_forward(opt.seed, opt.J, opt.spins, opt.beta, opt.h, opt.alpha, 0, opt.sweeps, opt.tape, stream)
        dmc_loss(opt.spins, opt.target, opt.gs, opt.loss, stream)
        dmc_backward(opt.seed, opt.J, opt.spins, opt.tape, opt.beta, opt.h, opt.alpha, 0, opt.sweeps, opt.gs,
                     opt.gJ, stream)
        out.append((float(T), float(opt.gJ.abs().mean()), float(opt.loss.mean())))
    return out


class SpinOptimizer:
    """Energy minimisation over the spin values (Sec. "Optimization of the spin
    values") for B lattices with per-bond couplings J [B, 2, L, L] (J = 1: the
    ferromagnet; random +-1: a spin glass).  Three methods:

    * anneal: Metropolis sweeps (the relaxed update with alpha -> infinity) at
      increasing beta;
    * gradient: s <- discretise(clip(s - eta sign(dE/ds), -1, 1)), all sites at once;
    * dmc: the spins are the parameters of the differentiable Monte Carlo
      loss E(F(s)), F the relaxed sweeps of Alg. 2; each iteration
      s <- discretise(clip(s - eta sign(d E(F(s)) / ds), -1, 1)), and the state
      the simulation produced is discretise(F(s)).

    Each method returns the energy per spin after every iteration (numpy).
    """

    def __init__(self, J, spins, h=0.0, seed=0):
        self.J = J.contiguous()
        self.spins = spins.clone().contiguous()
        self.B, self.L = spins.shape[0], spins.shape[-1]
        self.h, self.seed, self.sweep = h, seed, 0
        self.energy = torch.zeros(self.B, dtype=torch.float64, device=spins.device)
        self.grad = torch.zeros_like(self.spins)

    def _trace(self, rows):
        return (torch.stack(rows) / (self.L * self.L)).cpu().numpy()

    def anneal(self, betas, sweeps_per_beta, stream=None):
        tape = torch.empty(dmc_tape_floats(self.B, self.L, sweeps_per_beta), dtype=torch.float32,
                           device=self.spins.device)
        rows = []
        for beta in betas:
            dmc_forward(self.seed, self.J, self.spins, beta, self.h, 1e30, self.sweep, sweeps_per_beta, tape, stream)
            self.sweep += sweeps_per_beta
            dmc_energy(self.J, self.spins, self.h, self.energy, None, stream)
            rows.append(self.energy.clone())
        return self._trace(rows)

    def gradient(self, steps, eta=2.0, stream=None):
        rows = []
        for _ in range(steps):
            dmc_energy(self.J, self.spins, self.h, self.energy, self.grad, stream)
            dmc_spin_step(self.spins, self.grad, eta, stream)
            dmc_discretize(self.spins, stream)
            dmc_energy(self.J, self.spins, self.h, self.energy, None, stream)
            rows.append(self.energy.clone())
        return self._trace(rows)

    def dmc(self, steps, beta, alpha, eta=2.0, sweeps=1, stream=None, fused=True):
        if fused and sweeps <= dmc_spin_iter_max_sweeps(self.L):
            rows = []
            for _ in range(steps):
                dmc_spin_iter(self.seed, self.J, self.spins, self.energy, beta, self.h, alpha, eta, self.sweep,
                              sweeps, stream)
                self.sweep += sweeps
                rows.append(self.energy.clone())
            return self._trace(rows)
        tape = torch.empty(dmc_tape_floats(self.B, self.L, sweeps), dtype=torch.float32, device=self.spins.device)
        relaxed = torch.empty_like(self.spins)
        gJ = torch.empty_like(self.J)
        rows = []
        for _ in range(steps):
            relaxed.copy_(self.spins)
            dmc_forward(self.seed, self.J, relaxed, beta, self.h, alpha, self.sweep, sweeps, tape, stream)
            dmc_energy(self.J, relaxed, self.h, self.energy, self.grad, stream)
            dmc_backward(self.seed, self.J, relaxed, tape, beta, self.h, alpha, self.sweep, sweeps, self.grad, gJ,
                         stream)
            self.sweep += sweeps
            dmc_spin_step(self.spins, self.grad, eta, stream)
            dmc_discretize(self.spins, stream)
            dmc_discretize(relaxed, stream)
            dmc_energy(self.J, relaxed, self.h, self.energy, None, stream)
            rows.append(self.energy.clone())
        return self._trace(rows)

"""Differentiable Monte Carlo pattern optimisation (Alg. 2; Sec.
"Optimization of the exchange parameters").

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

from . import (adam, dmc_backward, dmc_discretize, dmc_forward, dmc_loss, dmc_step, dmc_step_max_sweeps,
               dmc_tape_floats)


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

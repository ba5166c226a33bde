"""GPU parity of the differentiable Monte Carlo kernels (Alg. 2) against the
float64 oracle.

Tolerance.  The kernels compute in float32 (the paper's PyTorch arithmetic;
expf is CUDA's, within 2 ulp).  Each sub-step evaluates about ten float
operations per site, so it injects a relative rounding error of order
10 eps32 (eps32 = 2^-24); later sub-steps propagate earlier errors with the
trajectory's own sensitivity.  That sensitivity is measured on the oracle by
perturbing the start spins by 1e-9 and recording the largest growth `cond` of
the difference over the run (a finite-difference condition number), so the
bound used below is  tol = 10 eps32 * n_substeps * max(cond, 1) * scale  (scale
the largest magnitude of the compared quantity), with a factor 4 of margin.
Integer-valued results (discretisation) and the loss gradient -2 (t - s) are
exact.
"""
import numpy as np
import pytest
import torch

import paper_2304_01772_gb300 as sm
from oracle import dmc as odmc
from paper_2304_01772_gb300 import dmc as pdmc

pytestmark = pytest.mark.gpu

SEED = 0x5EEDD3C0FFEE
EPS32 = 2.0 ** -24


def f32(x):
    return float(np.float32(x))


def make_case(B, L, seed):
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, size=(B, 2, L, L)).astype(np.float32)
    s0 = rng.uniform(-1, 1, size=(B, L, L)).astype(np.float32)
    target = rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)
    return J, s0, target


def oracle_run(J, s0, beta, h, alpha, lat, sweep0, n):
    s = s0.astype(np.float64).copy()
    tape = odmc.run(s, J.astype(np.float64), beta, h, alpha, SEED, lat, sweep0, n, tape=True)
    return s, tape


def condition(J, s0, beta, h, alpha, lat, sweep0, n):
    base, _ = oracle_run(J, s0, beta, h, alpha, lat, sweep0, n)
    d = 1e-9
    pert = s0.astype(np.float64) + d * np.random.default_rng(lat).choice([-1.0, 1.0], size=s0.shape)
    s = pert.copy()
    odmc.run(s, J.astype(np.float64), beta, h, alpha, SEED, lat, sweep0, n)
    return float(np.abs(s - base).max() / d)


@pytest.mark.parametrize("B,L,n,alpha", [(3, 8, 3, 4.0), (2, 16, 2, 2.0), (2, 64, 2, 4.0), (5, 32, 1, 10.0)])
def test_forward_and_tape_match_oracle(B, L, n, alpha):
    beta, h = f32(0.8), f32(0.05)
    J, s0, _ = make_case(B, L, 11 * L + n)
    spins = torch.from_numpy(s0.copy()).cuda()
    Jd = torch.from_numpy(J).cuda()
    tape = torch.full((sm.dmc_tape_floats(B, L, n),), np.nan, dtype=torch.float32, device="cuda")
    sm.dmc_forward(SEED, Jd, spins, beta, h, alpha, 7, n, tape)
    got = spins.cpu().numpy()
    gtape = tape.cpu().numpy().reshape(B, 2 * n, L * L // 2)
    for b in range(B):
        ref, rtape = oracle_run(J[b], s0[b], beta, h, alpha, b, 7, n)
        cond = condition(J[b], s0[b], beta, h, alpha, b, 7, n)
        tol = 4 * 10 * EPS32 * 2 * n * max(cond, 1.0)
        err = np.abs(got[b] - ref).max()
        assert err <= tol, (b, err, tol, cond)
        # tape: old values of the active sites of each sub-step, compressed order
        for k in range(2 * n):
            c = k & 1
            flat = rtape[k].reshape(-1)
            active = np.array([y * L + x for y in range(L) for x in range(L) if (x + y) % 2 == c])
            assert np.abs(gtape[b, k] - flat[active]).max() <= tol, (b, k)


@pytest.mark.parametrize("B,L,n,alpha", [(2, 8, 2, 3.0), (2, 32, 2, 4.0), (1, 64, 1, 4.0)])
def test_backward_matches_oracle(B, L, n, alpha):
    beta, h = f32(0.7), f32(-0.1)
    J, s0, target = make_case(B, L, 5 * L + n)
    spins = torch.from_numpy(s0.copy()).cuda()
    Jd = torch.from_numpy(J).cuda()
    tape = torch.empty(sm.dmc_tape_floats(B, L, n), dtype=torch.float32, device="cuda")
    sm.dmc_forward(SEED, Jd, spins, beta, h, alpha, 0, n, tape)
    gs = torch.empty_like(spins)
    loss = torch.empty(B, dtype=torch.float64, device="cuda")
    sm.dmc_loss(spins, torch.from_numpy(target).cuda(), gs, loss)
    gJ = torch.full_like(Jd, np.nan)
    sm.dmc_backward(SEED, Jd, spins, tape, beta, h, alpha, 0, n, gs, gJ)
    got_gs, got_gJ, got_loss = gs.cpu().numpy(), gJ.cpu().numpy(), loss.cpu().numpy()
    for b in range(B):
        ref, rtape = oracle_run(J[b], s0[b], beta, h, alpha, b, 0, n)
        rloss, rg = odmc.loss(ref, target[b])
        rgs, rgJ = odmc.backward(rtape, J[b].astype(np.float64), rg, beta, h, alpha, SEED, b, 0)
        cond = condition(J[b], s0[b], beta, h, alpha, b, 0, n)
        tol = 4 * 10 * EPS32 * 2 * n * max(cond, 1.0)
        assert abs(got_loss[b] - rloss) <= tol * (1 + rloss) * 4, (b, got_loss[b], rloss)
        assert np.abs(got_gJ[b] - rgJ).max() <= tol * max(1.0, np.abs(rgJ).max()) * 4, b
        assert np.abs(got_gs[b] - rgs).max() <= tol * max(1.0, np.abs(rgs).max()) * 4, b


def test_loss_gradient_and_discretisation_are_exact():
    rng = np.random.default_rng(9)
    s = rng.uniform(-1, 1, size=(4, 8, 8)).astype(np.float32)
    s[0, 0, :4] = [0.0, -0.0, 1e-30, -1e-30]
    t = rng.choice([-1.0, 1.0], size=s.shape).astype(np.float32)
    sd, td = torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda()
    g = torch.empty_like(sd)
    loss = torch.empty(4, dtype=torch.float64, device="cuda")
    sm.dmc_loss(sd, td, g, loss)
    np.testing.assert_array_equal(g.cpu().numpy(), np.float32(-2.0) * (t - s))
    ref = ((t.astype(np.float64) - s.astype(np.float64)) ** 2).reshape(4, -1).sum(1)
    np.testing.assert_allclose(loss.cpu().numpy(), ref, rtol=1e-6)
    sm.dmc_discretize(sd)
    np.testing.assert_array_equal(sd.cpu().numpy(), np.where(s < 0, -1.0, 1.0).astype(np.float32))


def test_pattern_optimisation_lowers_the_loss():
    """Alg. 2 as a training loop: the couplings steer lattices that start all
    up towards striped targets (Sec. Optimization of the exchange parameters).
    One relaxed sweep per iteration at T = 0.9, alpha = 10; the float64 oracle
    running the same loop on one 32^2 lattice lowers the loss about tenfold in
    150 iterations."""
    B, L = 16, 32
    y = np.arange(L)[:, None] * np.ones((1, L))
    target = np.stack([np.where(((y // (2 + b % 4)) % 2) == 0, 1.0, -1.0) for b in range(B)]).astype(np.float32)
    opt = pdmc.PatternOptimizer(torch.from_numpy(target).cuda(), beta=1 / 0.9, alpha=10.0, sweeps=1,
                                seed=3, lr=5e-2)
    hist = [opt.step().cpu().numpy().mean() for _ in range(150)]
    first, last = np.mean(hist[:15]), np.mean(hist[-15:])
    print(f"mean relaxed loss per lattice: first 15 iterations {first:.0f}, last 15 {last:.0f}")
    assert last < 0.3 * first


@pytest.mark.parametrize("B,L,K", [(4, 64, 1), (3, 32, 3), (2, 8, 2)])
def test_fused_step_equals_the_separate_calls(B, L, K):
    """spin_dmc_step (one launch, tape on chip) against forward + loss +
    reverse pass + Adam + discretisation: same kernels' arithmetic, so the
    spins, couplings and Adam moments agree bit for bit."""
    rng = np.random.default_rng(L + K)
    target = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)).cuda()
    start = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)).cuda()
    runs = []
    for fused in (True, False):
        opt = pdmc.PatternOptimizer(target, beta=1 / 0.9, alpha=10.0, sweeps=K, seed=7, lr=5e-2, spins=start,
                                    fused=fused)
        assert opt.fused == fused
        losses = [opt.step().cpu().numpy().copy() for _ in range(3)]
        runs.append((opt, losses))
    (a, la), (b, lb) = runs
    for name in ("spins", "J", "m", "v"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    np.testing.assert_allclose(np.array(la), np.array(lb), rtol=1e-12)


def test_energy_and_spin_step_kernels_are_exact_on_spin_glass_states():
    """+-1 spins and +-1 bonds: energies are integers (float64 sums exact),
    gradients small integers, the clipped sign step exact."""
    B, L, h = 3, 16, 0.0
    rng = np.random.default_rng(21)
    J = rng.choice([-1.0, 1.0], size=(B, 2, L, L)).astype(np.float32)
    s = rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)
    Jd, sd = torch.from_numpy(J).cuda(), torch.from_numpy(s.copy()).cuda()
    energy = torch.empty(B, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(sd)
    sm.dmc_energy(Jd, sd, h, energy, grad)
    for b in range(B):
        E, g = odmc.energy(s[b].astype(np.float64), J[b].astype(np.float64), h)
        assert energy[b].item() == E
        np.testing.assert_array_equal(grad[b].cpu().numpy(), g.astype(np.float32))
    sm.dmc_spin_step(sd, grad, 2.0)
    for b in range(B):
        np.testing.assert_array_equal(sd[b].cpu().numpy(),
                                      odmc.spin_step(s[b].astype(np.float64), grad[b].cpu().numpy(), 2.0))


def test_spin_value_optimisation_three_methods():
    """+-J spin glass, 16 lattices of 32^2 from random states: annealed
    Metropolis gets close to the ground-state energy per spin (about -1.40
    for the 2D +-J model), the gradient-only method stops higher, and the
    differentiable Monte Carlo reaches lower energies than the gradient
    (the ordering reported in Sec. Optimization of the spin values)."""
    B, L = 16, 32
    rng = np.random.default_rng(8)
    J = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, 2, L, L)).astype(np.float32)).cuda()
    s0 = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)).cuda()
    mc = pdmc.SpinOptimizer(J, s0, seed=1).anneal(np.linspace(0.1, 3.0, 30), 5)
    gd = pdmc.SpinOptimizer(J, s0, seed=1).gradient(50, eta=2.0)
    dm = pdmc.SpinOptimizer(J, s0, seed=1).dmc(60, beta=2.0, alpha=10.0, eta=2.0)
    e_mc, e_gd, e_dm = mc[-1].mean(), gd[-1].mean(), dm.min(axis=0).mean()
    print(f"energy per spin: annealing {e_mc:.3f}, gradient {e_gd:.3f}, DMC (best) {e_dm:.3f}")
    assert e_mc < -1.3
    assert e_dm < e_gd - 0.1
    assert e_gd < -0.8


@pytest.mark.parametrize("L,K", [(64, 1), (32, 3)])
def test_fused_spin_iteration_equals_the_separate_calls(L, K):
    B = 4
    rng = np.random.default_rng(L * K)
    J = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, 2, L, L)).astype(np.float32)).cuda()
    s0 = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)).cuda()
    a = pdmc.SpinOptimizer(J, s0, seed=5)
    b = pdmc.SpinOptimizer(J, s0, seed=5)
    ea = a.dmc(4, beta=2.0, alpha=10.0, sweeps=K, fused=True)
    eb = b.dmc(4, beta=2.0, alpha=10.0, sweeps=K, fused=False)
    assert torch.equal(a.spins, b.spins)
    np.testing.assert_array_equal(ea, eb)


def test_benchmark_shape_sampled():
    """The benchmark's shape (1024 lattices of 64^2, one relaxed sweep per
    iteration) in the fused launch it times: equal bit for bit to the separate
    calls at full size, and the relaxed forward pass of sampled lattices within
    the oracle's tolerance above."""
    B, L, K = 1024, 64, 1
    rng = np.random.default_rng(2024)
    target = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)).cuda()
    start = torch.from_numpy(rng.choice([-1.0, 1.0], size=(B, L, L)).astype(np.float32)).cuda()
    runs = []
    for fused in (True, False):
        opt = pdmc.PatternOptimizer(target, beta=1 / 0.9, alpha=10.0, sweeps=K, seed=7, lr=5e-2, spins=start,
                                    fused=fused)
        for _ in range(2):
            opt.step()
        runs.append(opt)
    for name in ("spins", "J", "m", "v"):
        assert torch.equal(getattr(runs[0], name), getattr(runs[1], name)), name
    beta, h, alpha = f32(0.8), f32(0.05), 4.0
    J, s0, _ = make_case(B, L, 99)
    spins = torch.from_numpy(s0.copy()).cuda()
    tape = torch.empty((sm.dmc_tape_floats(B, L, K),), dtype=torch.float32, device="cuda")
    sm.dmc_forward(SEED, torch.from_numpy(J).cuda(), spins, beta, h, alpha, 3, K, tape)
    got = spins.cpu().numpy()
    for b in (0, 517, 1023):
        ref, _ = oracle_run(J[b], s0[b], beta, h, alpha, b, 3, K)
        cond = condition(J[b], s0[b], beta, h, alpha, b, 3, K)
        tol = 4 * 10 * EPS32 * 2 * K * max(cond, 1.0)
        assert np.abs(got[b] - ref).max() <= tol, b


def test_gradient_by_temperature_matches_the_oracle():
    """The temperature study (coupling-gradient size for one relaxed sweep from
    the ordered start, per T) on the GPU against the float64 oracle, and its
    maximum at an intermediate temperature."""
    L = 16
    y = np.arange(L)[:, None] * np.ones((1, L))
    pats = ([np.where((y // w) % 2 == 0, 1.0, -1.0) for w in (2, 3, 4)] +
            [np.where((y.T // w) % 2 == 0, 1.0, -1.0) for w in (2, 3)])
    target = torch.from_numpy(np.array(pats, dtype=np.float32)).cuda()
    Ts = [0.5, 1.0, 2.0, 4.0, 6.0, 10.0, 30.0, 100.0]
    got = pdmc.gradient_by_temperature(target, Ts, alpha=10.0, sweeps=1, seed=SEED)
    sizes = [g for _, g, _ in got]
    k = int(np.argmax(sizes))
    assert 0 < k < len(Ts) - 1, sizes
    for T, g, _ in got:
        ref = []
        for b, t in enumerate(pats):
            s = np.ones((L, L))
            J = np.ones((2, L, L))
            beta = f32(1.0 / T)
            tape = odmc.run(s, J, beta, 0.0, 10.0, SEED, b, 0, 1, tape=True)
            _, gs = odmc.loss(s, t)
            _, gJ = odmc.backward(tape, J, gs, beta, 0.0, 10.0, SEED, b, 0)
            ref.append(gJ)
        want = float(np.abs(np.array(ref)).mean())
        assert abs(g - want) <= 1e-4 * max(want, 1e-3), (T, g, want)

"""Pins of the differentiable Monte Carlo oracle (Alg. 2) against facts that
do not come from the oracle itself:

* its reverse pass against central finite differences of its forward pass
  (the forward is smooth in J and s for fixed random numbers);
* alpha -> infinity: the relaxed update on +-1 spins becomes Metropolis with
  acceptance r < exp(-beta dE), checked against a plain chain written here
  whose dE is a brute-force difference of the per-bond Hamiltonian
  H = -sum J_ij s_i s_j - h sum s_i (this also pins the bond orientation);
* J = h = 0: every active site moves to s (1 - 2 sigma(alpha (1 - r)));
* |s| never grows: |1 - 2q| <= 1.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import dmc

SEED = 0x0DDC0FFEE


def r_of(seed, lattice, sweep, colour, L, x, y):
    """The site's uniform: Philox lane of the Ising layout, top 24 bits."""
    k = (y * L + x) >> 1
    u = oracle.philox4x32_10([k >> 2, lattice, sweep, colour], [seed & 0xFFFFFFFF, seed >> 32])[k & 3]
    return float(int(u) >> 8) / 2 ** 24


def hamiltonian(s, J, h):
    L = s.shape[0]
    H = 0.0
    for y in range(L):
        for x in range(L):
            H -= J[0, y, x] * s[y, x] * s[y, (x + 1) % L]
            H -= J[1, y, x] * s[y, x] * s[(y + 1) % L, x]
            H -= h * s[y, x]
    return H


def rand_case(L, seed, relaxed=True):
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, size=(2, L, L))
    s = rng.uniform(-1, 1, size=(L, L)) if relaxed else rng.choice([-1.0, 1.0], size=(L, L))
    target = rng.choice([-1.0, 1.0], size=(L, L))
    return J, s, target


def loss_after(J, s0, target, beta, h, alpha, n_sweeps):
    s = s0.copy()
    dmc.run(s, J, beta, h, alpha, SEED, 3, 5, n_sweeps)
    return dmc.loss(s, target)[0]


def test_reverse_pass_matches_finite_differences():
    L, n_sweeps, beta, h, alpha = 6, 2, 0.8, 0.1, 3.0
    J, s0, target = rand_case(L, 1)
    s = s0.copy()
    tape = dmc.run(s, J, beta, h, alpha, SEED, 3, 5, n_sweeps, tape=True)
    _, g = dmc.loss(s, target)
    gs0, gJ = dmc.backward(tape, J, g, beta, h, alpha, SEED, 3, 5)
    eps = 1e-6
    fd = np.zeros_like(J)
    for idx in np.ndindex(J.shape):
        Jp, Jm = J.copy(), J.copy()
        Jp[idx] += eps
        Jm[idx] -= eps
        fd[idx] = (loss_after(Jp, s0, target, beta, h, alpha, n_sweeps) -
                   loss_after(Jm, s0, target, beta, h, alpha, n_sweeps)) / (2 * eps)
    np.testing.assert_allclose(gJ, fd, rtol=1e-5, atol=1e-7 * np.abs(fd).max())
    fs = np.zeros_like(s0)
    for idx in [(0, 0), (1, 4), (5, 5), (3, 2)]:
        sp, sm = s0.copy(), s0.copy()
        sp[idx] += eps
        sm[idx] -= eps
        fs[idx] = (loss_after(J, sp, target, beta, h, alpha, n_sweeps) -
                   loss_after(J, sm, target, beta, h, alpha, n_sweeps)) / (2 * eps)
        assert abs(gs0[idx] - fs[idx]) <= 1e-5 * max(1.0, abs(fs[idx])), (idx, gs0[idx], fs[idx])


def test_alpha_infinity_is_metropolis_on_the_bond_hamiltonian():
    L, beta, h = 8, 0.45, 0.07
    J, s0, _ = rand_case(L, 2, relaxed=False)
    s = s0.copy()
    dmc.run(s, J, beta, h, 1e300, SEED, 0, 0, 3)
    ref = s0.copy()
    for t in range(3):
        for c in range(2):
            old = ref.copy()
            for y in range(L):
                for x in range(L):
                    if (x + y) % 2 != c:
                        continue
                    flipped = old.copy()
                    flipped[y, x] = -flipped[y, x]
                    dE = hamiltonian(flipped, J, h) - hamiltonian(old, J, h)
                    if r_of(SEED, 0, t, c, L, x, y) < math.exp(-beta * dE):
                        ref[y, x] = -old[y, x]
    assert set(np.unique(s)) <= {-1.0, 1.0}
    np.testing.assert_array_equal(s, ref)


def test_zero_couplings_closed_form():
    L, alpha = 6, 4.0
    J = np.zeros((2, L, L))
    s = np.random.default_rng(3).uniform(-1, 1, size=(L, L))
    before = s.copy()
    dmc.substep(s, J, 0.7, 0.0, alpha, SEED, 1, 9, 1)
    for y in range(L):
        for x in range(L):
            if (x + y) % 2 == 1:
                q = 1.0 / (1.0 + math.exp(-alpha * (1.0 - r_of(SEED, 1, 9, 1, L, x, y))))
                assert s[y, x] == pytest.approx(before[y, x] * (1 - 2 * q), rel=1e-14, abs=1e-15)
            else:
                assert s[y, x] == before[y, x]


def test_relaxed_spins_never_grow():
    L = 10
    rng = np.random.default_rng(4)
    J = rng.uniform(-1.5, 1.5, size=(2, L, L))
    s = rng.uniform(-1, 1, size=(L, L))
    for t in range(6):
        for c in range(2):
            before = np.abs(s).copy()
            dmc.substep(s, J, 1.2, -0.2, 8.0, SEED, 0, t, c)
            assert np.all(np.abs(s) <= before + 1e-15)


def test_loss_and_discretisation():
    s = np.array([[0.3, -0.2], [0.0, -1.0]])
    t = np.array([[1.0, -1.0], [-1.0, 1.0]])
    v, g = dmc.loss(s, t)
    assert v == pytest.approx(0.49 + 0.64 + 1.0 + 4.0)
    np.testing.assert_allclose(g, -2 * (t - s))
    np.testing.assert_array_equal(dmc.discretize(s), [[1.0, -1.0], [1.0, -1.0]])


def test_energy_matches_the_bond_hamiltonian_and_its_gradient():
    L, h = 6, 0.3
    rng = np.random.default_rng(5)
    J = rng.choice([-1.0, 1.0], size=(2, L, L))
    s = rng.uniform(-1, 1, size=(L, L))
    E, g = dmc.energy(s, J, h)
    assert E == pytest.approx(hamiltonian(s, J, h), rel=1e-13)
    eps = 1e-6
    for idx in [(0, 0), (2, 5), (5, 1), (3, 3)]:
        sp, sm = s.copy(), s.copy()
        sp[idx] += eps
        sm[idx] -= eps
        fd = (hamiltonian(sp, J, h) - hamiltonian(sm, J, h)) / (2 * eps)
        assert g[idx] == pytest.approx(fd, rel=1e-7, abs=1e-8)


def test_spin_step_is_a_clipped_sign_step():
    s = np.array([[0.9, -0.5], [0.0, -1.0]])
    g = np.array([[-1.0, 2.0], [0.0, -0.1]])
    np.testing.assert_array_equal(dmc.spin_step(s, g, 0.5), [[1.0, -1.0], [0.0, -0.5]])


def _stripes(L, widths=(2, 3, 4)):
    y = np.arange(L)[:, None] * np.ones((1, L))
    return ([np.where((y // w) % 2 == 0, 1.0, -1.0) for w in widths] +
            [np.where((y.T // w) % 2 == 0, 1.0, -1.0) for w in widths[:2]])


def _grad_size(T, J0, L=16, alpha=10.0, seed=7):
    """Mean |dL/dJ| of one relaxed sweep from all +1 with couplings J0 (the
    temperature study of Sec. "Optimization of the exchange parameters")."""
    out = []
    for b, t in enumerate(_stripes(L)):
        s = np.ones((L, L))
        J = np.full((2, L, L), J0)
        tape = dmc.run(s, J, 1.0 / T, 0.0, alpha, seed, b, 0, 1, tape=True)
        _, g = dmc.loss(s, t)
        _, gJ = dmc.backward(tape, J, g, 1.0 / T, 0.0, alpha, seed, b, 0)
        out.append(gJ)
    return np.abs(np.array(out)).mean()


def test_gradient_size_depends_on_temperature_through_beta_J():
    """With h = 0 the relaxed dynamics depend on beta J only: doubling T and the
    couplings gives the same trajectory (same draws, same acceptance values) and
    halves dL/dJ exactly -- in binary floating point, since the factor is a
    power of two.  A misplaced beta or J in the forward or reverse pass breaks
    this."""
    for T in (0.7, 2.0, 5.0):
        assert _grad_size(2 * T, 2.0) == _grad_size(T, 1.0) / 2


def test_gradient_size_peaks_at_an_intermediate_temperature():
    """From the ordered start the gradient vanishes at low T (nothing moves)
    and at high T (the moves no longer depend on the couplings); it is largest
    in between, the behaviour the paper reports for its pattern optimisation."""
    Ts = [0.5, 1.0, 2.0, 4.0, 6.0, 10.0, 30.0, 100.0]
    g = [_grad_size(T, 1.0) for T in Ts]
    k = int(np.argmax(g))
    assert 0 < k < len(Ts) - 1, g
    assert g[0] < 0.01 * g[k] and g[-1] < 0.1 * g[k], g

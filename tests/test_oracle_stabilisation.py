"""Pins of the oracle's momentum stabilisation (Sec. 4.1: the mean velocity of
the whole domain is subtracted from the velocity in the equilibrium).

In a fully periodic box without obstacles the collision changes a cell's
momentum by -omega_odd (j - rho0 (u - ubar)) (the odd part relaxes towards
3 w rho0 c.(u - ubar)), streaming moves momentum without changing it, and the
mean of u - ubar over the fluid cells is zero.  So the total momentum J obeys
J_{n+1} = (1 - omega_odd) J_n exactly, for any state; without stabilisation
J is conserved.  A uniform flow stays uniform and decays by the same factor
per step.  A state whose mean velocity is zero is not changed by switching
the stabilisation on.
"""
import numpy as np
import pytest

import oracle
from lbm_inputs import Lattice

Q = 19


def total_momentum(sim):
    _, u, fl, _, _ = sim.fields()
    return u[:, fl == 0].sum(axis=1)


def random_state(lat, seed, mean=(0.0, 0.0, 0.0)):
    rng = np.random.default_rng(seed)
    c, w, _ = oracle.lattice_tables()
    n = lat.ncells
    u = np.asarray(mean)[:, None] + 0.01 * rng.standard_normal((3, n))
    rho = 1.0 + 0.01 * rng.standard_normal(n)
    cu = c @ u
    uu = (u * u).sum(axis=0)
    f = w[:, None] * (rho[None, :] + 3 * cu + 4.5 * cu * cu - 1.5 * uu[None, :])
    return f + 1e-4 * rng.standard_normal(f.shape)


@pytest.mark.parametrize("tau", [0.7, 1.3, 6.0])
def test_total_momentum_decays_by_one_minus_omega_odd(tau):
    lat = Lattice(10, 9, 8, tau=tau, periodic=(1, 1, 1))
    s = oracle.Sim(lat)
    s.set_pdfs(random_state(lat, 1, mean=(0.02, -0.01, 0.015)))
    s.set_momentum_stabilisation(True)
    oo = oracle.omega_odd(tau, lat.magic)
    J = total_momentum(s)
    for _ in range(6):
        s.step(1)
        Jn = total_momentum(s)
        assert np.allclose(Jn, (1 - oo) * J, rtol=1e-11, atol=1e-14 * np.abs(J).max())
        J = Jn


def test_momentum_conserved_without_stabilisation():
    lat = Lattice(10, 9, 8, tau=0.9, periodic=(1, 1, 1))
    s = oracle.Sim(lat)
    s.set_pdfs(random_state(lat, 2, mean=(0.02, -0.01, 0.015)))
    J = total_momentum(s)
    s.step(5)
    assert np.allclose(total_momentum(s), J, rtol=1e-12)


def test_uniform_flow_stays_uniform_and_decays():
    lat = Lattice(6, 5, 7, tau=0.8, periodic=(1, 1, 1))
    s = oracle.Sim(lat)
    u0 = np.array([0.03, -0.02, 0.01])
    feq = oracle.equilibrium(1.0, u0)
    s.set_pdfs(np.repeat(feq[:, None], lat.ncells, axis=1))
    s.set_momentum_stabilisation(True)
    oo = oracle.omega_odd(0.8, lat.magic)
    s.step(5)
    _, u, _, _, _ = s.fields()
    assert np.allclose(u, ((1 - oo) ** 5 * u0)[:, None], rtol=1e-11, atol=1e-16)


def test_uniform_flow_one_step_closed_form():
    """From f = f^eq(rho0, u0) everywhere: ubar = u0, so both equilibrium
    parts are taken at zero velocity: f1 = f - omega (f^e - w rho0)
    - omega_odd f^o, with f^e - w rho0 = w rho0 (4.5 (c.u0)^2 - 1.5 u0^2) and
    f^o = 3 w rho0 c.u0 (streaming leaves a uniform state unchanged)."""
    tau = 0.8
    lat = Lattice(5, 4, 6, tau=tau, periodic=(1, 1, 1))
    s = oracle.Sim(lat)
    u0 = np.array([0.03, -0.02, 0.01])
    c, w, _ = oracle.lattice_tables()
    feq = oracle.equilibrium(1.0, u0)
    s.set_pdfs(np.repeat(feq[:, None], lat.ncells, axis=1))
    s.set_momentum_stabilisation(True)
    s.step(1)
    om, oo = 1 / tau, oracle.omega_odd(tau, lat.magic)
    cu = c @ u0
    f1 = feq - om * w * (4.5 * cu * cu - 1.5 * u0 @ u0) - oo * 3 * w * cu
    pdfs = s.fields()[4]
    assert np.allclose(pdfs, f1[:, None], rtol=0, atol=1e-16)


def test_zero_mean_state_unchanged_by_stabilisation():
    lat = Lattice(12, 10, 8, tau=0.9, periodic=(1, 1, 1))
    f = random_state(lat, 3)
    # remove the mean momentum exactly: mirror the state in x, y, z and average
    c, _, opp = oracle.lattice_tables()
    n = lat.ncells
    idx = np.arange(n)
    i, j, k = idx % 12, (idx // 12) % 10, idx // 120
    mirror = ((-i) % 12) + 12 * (((-j) % 10) + 10 * ((-k) % 8))
    f = 0.5 * (f + f[opp][:, mirror])
    a, b = oracle.Sim(lat), oracle.Sim(lat)
    a.set_pdfs(f)
    b.set_pdfs(f)
    assert np.abs(total_momentum(a)).max() < 1e-15
    b.set_momentum_stabilisation(True)
    a.step(4)
    b.step(4)
    assert np.allclose(a.fields()[1], b.fields()[1], rtol=0, atol=1e-15)


def test_collision_with_own_velocity_as_mean_relaxes_odd_part_to_zero():
    f = random_state(Lattice(1, 1, 1), 4, mean=(0.02, 0.01, -0.01))[:, 0]
    c, _, opp = oracle.lattice_tables()
    u = c.T @ f
    oo, om = 1.4, 0.9
    ft = oracle.collide_cell(f, om, oo, 1.0, ubar=u)
    fo, fto = 0.5 * (f - f[opp]), 0.5 * (ft - ft[opp])
    assert np.allclose(fto, (1 - oo) * fo, rtol=0, atol=1e-16)

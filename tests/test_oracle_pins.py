"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU).  None re-types an oracle formula and
compares it with itself: each checks a closed form, an invariant, a special
case, a printed table value or a brute-force enumeration.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from lbm_inputs import (Lattice, Particle, SplitMix64, quat_from_axis, shear_lattice,
                        small_shear, axis_from_quat)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sig(x, d):
    return float(f"{x:.{d}g}")


# --------------------------------------------------------------------------
# closed forms against the paper's printed numbers
# --------------------------------------------------------------------------

def test_table_A_tirado_rows():
    """Tirado coefficients reproduce the appendix table's reference rows."""
    g = json.load(open(os.path.join(GOLDEN, "table_A_tirado.json")))
    r, mu, F = g["radius_m"], g["mu"], g["force_z_N"]
    for i, inv_eps in enumerate(g["inverse_eps"]):
        Lw = inv_eps * r            # full spherocylinder length (with caps)
        Ln = Lw - 2.0 * r           # without caps
        M = g["torque_x_1e-15"][i] * 1e-15
        for L, tag in ((Lw, "wC"), (Ln, "nC")):
            gp, gq, gr = cf.tirado_coefficients(mu, L, r)
            assert round(F / gp * 1e6) == g[f"U_par_Tir_{tag}_um_s"][i]
            assert round(F / gq * 1e6) == g[f"U_perp_Tir_{tag}_um_s"][i]
            assert _sig(M / gr, 3) == pytest.approx(g[f"omega_Tir_{tag}_1_s"][i], rel=1e-9)


def test_unit_conversion_examples():
    g = json.load(open(os.path.join(GOLDEN, "unit_conversion.json")))
    for c in g["cases"]:
        dt = cf.lattice_time_step(c["tau"], c["dx_m"], c["nu_m2_s"])
        assert _sig(dt, c["printed_digits"]) == pytest.approx(c["dt_s"], rel=1e-12)


# --------------------------------------------------------------------------
# lattice, equilibrium, collision
# --------------------------------------------------------------------------

def test_d3q19_isotropy():
    """Weights and velocities give the lattice tensors of D3Q19 with c_s^2 = 1/3."""
    c, w, opp = oracle.lattice_tables()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all(c[opp] == -c)
    d = np.eye(3)
    assert np.allclose(np.einsum("q,qa->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb->ab", w, c, c), d / 3.0, atol=1e-16)
    assert np.allclose(np.einsum("q,qa,qb,qc->abc", w, c, c, c), 0, atol=1e-16)
    t4 = np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(t4, iso, atol=1e-16)
    assert sorted(np.round(w * 36).astype(int).tolist()) == [1] * 12 + [2] * 6 + [12]


def test_magic_parameter_matches_paper_formula():
    """Lambda = 3/16 gives the paper's lambda_o = -8(2 - omega)/(8 - omega)."""
    for tau in (0.55, 0.8, 1.0, 1.7, 6.0):
        om = 1.0 / tau
        assert oracle.omega_odd(tau, 3.0 / 16.0) == pytest.approx(8 * (2 - om) / (8 - om), rel=1e-14)
    # tau = 0.8 worked through: omega = 1.25, omega_o = 8/9, Lambda = 0.3 * 0.625
    assert oracle.omega_odd(0.8, 3 / 16) == pytest.approx(8.0 / 9.0, rel=1e-15)


def test_equilibrium_moments():
    """Zeroth, first and second moments of the incompressible equilibrium:
    rho, rho0 u, rho/3 I + rho0 u u."""
    c, w, _ = oracle.lattice_tables()
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho = 1.0 + 0.1 * rng.standard_normal()
        rho0 = 1.0 + 0.2 * rng.random()
        u = 0.05 * rng.standard_normal(3)
        feq = oracle.equilibrium(rho, u, rho0)
        assert feq.sum() == pytest.approx(rho, abs=1e-15)
        assert np.allclose(c.T @ feq, rho0 * u, atol=1e-16)
        P = np.einsum("q,qa,qb->ab", feq, c, c)
        assert np.allclose(P, rho / 3 * np.eye(3) + rho0 * np.outer(u, u), atol=1e-15)


def test_collision_conserves_mass_and_momentum():
    c, w, _ = oracle.lattice_tables()
    rng = np.random.default_rng(7)
    for _ in range(20):
        f = w * (1.0 + 0.1 * rng.standard_normal(19))
        g = 1e-4 * rng.standard_normal(3)
        om, oo = 1.0 / 0.7, oracle.omega_odd(0.7, 3 / 16)
        ft = oracle.collide_cell(f, om, oo, 1.0)
        assert ft.sum() == pytest.approx(f.sum(), abs=1e-15)
        assert np.allclose(c.T @ ft, c.T @ f, atol=1e-16)
        # the body-force source adds rho0 g of momentum and no mass
        ftg = oracle.collide_cell(f, om, oo, 1.0, g)
        assert ftg.sum() == pytest.approx(f.sum(), abs=1e-15)
        assert np.allclose(c.T @ ftg - c.T @ f, g, atol=1e-16)


def test_trt_reduces_to_bgk_when_rates_equal():
    """With omega_odd = omega the TRT operator is BGK: f - omega (f - f^eq)."""
    _, w, _ = oracle.lattice_tables()
    rng = np.random.default_rng(9)
    c, _, _ = oracle.lattice_tables()
    for tau in (0.6, 1.0, 1.9):
        om = 1.0 / tau
        f = w * (1.0 + 0.2 * rng.standard_normal(19))
        ft = oracle.collide_cell(f, om, om, 1.0)
        feq = oracle.equilibrium(f.sum(), c.T @ f, 1.0)
        assert np.allclose(ft, f - om * (f - feq), atol=1e-16)


def test_trt_relaxes_even_and_odd_parts_separately():
    """Even and odd deviations from equilibrium decay by (1 - omega) and
    (1 - omega_odd) respectively, with pairs (q, opposite q) coupled."""
    c, w, opp = oracle.lattice_tables()
    rng = np.random.default_rng(11)
    f = w * (1.0 + 0.2 * rng.standard_normal(19))
    feq = oracle.equilibrium(f.sum(), c.T @ f, 1.0)
    om, oo = 1.0 / 0.9, 0.37
    ft = oracle.collide_cell(f, om, oo, 1.0)
    ne = 0.5 * ((f - feq) + (f - feq)[opp])
    no = 0.5 * ((f - feq) - (f - feq)[opp])
    assert np.allclose(ft - feq, (1 - om) * ne + (1 - oo) * no, atol=1e-16)


# --------------------------------------------------------------------------
# whole-lattice invariants and exact flows
# --------------------------------------------------------------------------

def _fill_equilibrium(sim, rho, u):
    feq = oracle.equilibrium(rho, u, 1.0)
    sim.set_pdfs(np.repeat(feq[:, None], sim.n, axis=1))


def test_uniform_flow_is_a_fixed_point():
    lat = Lattice(6, 5, 7, tau=0.7, periodic=(1, 1, 1))
    s = oracle.Sim(lat)
    u0 = np.array([0.013, -0.007, 0.021])
    _fill_equilibrium(s, 1.0, u0)
    s.step(10)
    rho, u, fl, pid, pdf = s.fields()
    assert np.allclose(u, u0[:, None], atol=1e-15, rtol=0)
    assert np.allclose(rho, 1.0, atol=1e-14, rtol=0)


@pytest.mark.parametrize("shape", [0, 1])
def test_body_translating_with_a_uniform_flow_is_a_fixed_point(shape):
    """Moving-obstacle bounce-back (Eq. LBMMovWall) returns f~_q - 6 w_q rho0
    c_q . u_s, and the equilibrium's odd part is exactly f^eq_qbar - f^eq_q =
    -6 w_q rho0 c_q . u: a body translating at U inside fluid at rest in the
    frame of U (uniform f^eq(rho0, U)) leaves every population unchanged.  The
    force vanishes too: the links in directions q and qbar of a closed body
    in a periodic box are equally many and carry equal even parts.  A wrong
    sign, factor or direction in the bounce-back breaks both."""
    lat = Lattice(16, 14, 12, tau=0.75, periodic=(1, 1, 1))
    U = np.array([0.03, -0.02, 0.01])
    t = np.array([0.6, 0.5, -0.3])
    body = Particle(pos=(7.3, 6.6, 5.9), quat=quat_from_axis(t / np.linalg.norm(t)), semi_axes=(4.5, 2.2, 2.2),
                    vel=tuple(U), fixed=1, shape=shape)
    s = oracle.Sim(lat, [body])
    _fill_equilibrium(s, 1.0, U)
    s.step(12)
    rho, u, fl, pid, pdf = s.fields()
    m = fl == 0
    assert (~m).sum() > 50
    feq = oracle.equilibrium(1.0, U, 1.0)
    assert np.abs(pdf[:, m] - feq[:, None]).max() < 1e-15
    F, M = s.forces()
    assert np.abs(F).max() < 1e-13 and np.abs(M).max() < 1e-12
    # the same body at rest in that flow is not a fixed point and feels drag along U
    s2 = oracle.Sim(lat, [Particle(pos=body.pos, quat=body.quat, semi_axes=body.semi_axes, fixed=1, shape=shape)])
    _fill_equilibrium(s2, 1.0, U)
    s2.step(1)
    F2, _ = s2.forces()
    assert F2[0] @ U > 1e-3 * np.linalg.norm(U)


def test_mass_conserved_with_moving_walls():
    lat = shear_lattice(12, 16, 10, 0.8, 0.03)
    s = oracle.Sim(lat)
    m0 = s.fields()[0].sum()
    s.step(200)
    m1 = s.fields()[0].sum()
    assert abs(m1 - m0) / m0 < 1e-13


@pytest.mark.parametrize("tau", [0.8, 1.5])
def test_couette_exact_linear_profile(tau):
    """Half-way moving walls: the steady profile is the exact line through
    -U_w at y = 0.5 and +U_w at y = ny - 1.5, for any tau."""
    ny, uw = 18, 0.01
    lat = shear_lattice(3, ny, 3, tau, uw)
    s = oracle.Sim(lat)
    nu = cf.lattice_viscosity(tau)
    H = ny - 2
    s.step(int(30 * H * H / (math.pi ** 2 * nu)))
    _, u, _, _, _ = s.fields()
    ux = u[0].reshape(3, ny, 3)[1, :, 1]
    y = np.arange(ny)
    ex = cf.couette_profile(y, ny, -uw, uw)
    assert np.abs(ux[1:-1] - ex[1:-1]).max() < 1e-10 * uw
    assert np.abs(u[1]).max() < 1e-14 and np.abs(u[2]).max() < 1e-14


def test_poiseuille_exact_with_magic_three_sixteenths():
    """Body-force driven channel: with Lambda = 3/16 the parabola with walls
    half-way is reproduced to round-off; Lambda = 1/4 misplaces the walls."""
    ny, g, tau = 16, 1e-6, 0.9
    nu = cf.lattice_viscosity(tau)
    y = np.arange(ny)
    ex = cf.poiseuille_profile(y, ny, g, nu)
    errs = {}
    for magic in (3.0 / 16.0, 0.25):
        lat = Lattice(3, ny, 3, tau=tau, magic=magic, periodic=(1, 0, 1), body_force=(g, 0, 0))
        s = oracle.Sim(lat)
        s.step(int(40 * (ny - 2) ** 2 / (math.pi ** 2 * nu)))
        _, u, _, _, _ = s.fields()
        ux = u[0].reshape(3, ny, 3)[1, :, 1]
        errs[magic] = np.abs(ux[1:-1] - ex[1:-1]).max() / ex.max()
    assert errs[3.0 / 16.0] < 1e-9
    assert errs[0.25] > 1e-4


# --------------------------------------------------------------------------
# particles: mapping, links, momentum exchange, rigid body
# --------------------------------------------------------------------------

def _brute_inside(rec, dims, periodic):
    """Cell-centre-in-ellipsoid mask by an independent route (scipy rotation)."""
    from scipy.spatial.transform import Rotation
    w, x, y, z = rec[3:7]
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = np.stack([i - rec[0], j - rec[1], k - rec[2]]).reshape(3, -1).astype(float)
    for a, n in enumerate(dims):
        if periodic[a]:
            d[a] -= n * np.round(d[a] / n)
    p = R.T @ d
    s = (p[0] / rec[13]) ** 2 + (p[1] / rec[14]) ** 2 + (p[2] / rec[15]) ** 2
    return s


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_obstacle_mapping_matches_bruteforce(seed):
    rng = SplitMix64(seed)
    lat = Lattice(28, 26, 24, periodic=(1, 0, 1))
    ps = [Particle(pos=(1.3 + 3 * seed, 12.6, 22.1), quat=quat_from_axis(rng.unit_vector()),
                   semi_axes=(7.5, 2.5, 2.0)),
          Particle(pos=(16.2, 11.7, 8.9), quat=quat_from_axis(rng.unit_vector()),
                   semi_axes=(6.0, 3.0, 3.0))]
    s = oracle.Sim(lat, ps)
    _, _, fl, pid, _ = s.fields()
    rec = oracle.particle_records(ps)
    masks = [_brute_inside(r, (28, 26, 24), (1, 0, 1)) for r in rec]
    fluid_region = np.ones(lat.ncells, bool)
    yy = np.repeat(np.arange(26)[None, :, None], 24, 0).repeat(28, 2).ravel()
    fluid_region[(yy == 0) | (yy == 25)] = False
    exp = np.full(lat.ncells, 0xFFFFFFFF, np.uint64)
    near = np.zeros(lat.ncells, bool)
    for p in (1, 0):
        exp[(masks[p] <= 1.0) & fluid_region] = p
        near |= np.abs(masks[p] - 1.0) < 1e-9
    ok = fluid_region & ~near
    assert np.all(pid[ok].astype(np.uint64) == exp[ok])
    assert np.all(fl[ok] == np.where(exp[ok] == 0xFFFFFFFF, 0, 2))
    assert np.all(fl[~fluid_region] == 1)


def test_mapped_volume_converges_to_ellipsoid_volume():
    rng = SplitMix64(4)
    vols = []
    for scale in (1.0, 2.0):
        a, b = 6.0 * scale, 2.5 * scale
        n = int(2 * a + 6)
        lat = Lattice(n, n, n, periodic=(1, 1, 1))
        p = Particle(pos=(n / 2 - 0.37, n / 2 + 0.21, n / 2 + 0.05),
                     quat=quat_from_axis(rng.unit_vector()), semi_axes=(a, b, b))
        s = oracle.Sim(lat, [p])
        _, _, fl, _, _ = s.fields()
        vols.append(abs((fl == 2).sum() / (4 / 3 * math.pi * a * b * b) - 1))
    assert vols[1] < 0.02


def test_links_match_enumeration():
    w = small_shear(seed=5, n=20)
    s = oracle.Sim(w.lattices[0], [_scaled(w.particles[0], 0.6)])
    cell, q, pid = s.links()
    _, _, fl, pidf, _ = s.fields()
    c, _, _ = oracle.lattice_tables()
    dims = (20, 20, 20)
    exp = []
    fl3 = fl.reshape(20, 20, 20)
    for idx in np.nonzero(fl == 0)[0]:
        i, j, k = idx % 20, (idx // 20) % 20, idx // 400
        for qq in range(1, 19):
            ii, jj, kk = (i + c[qq, 0]) % 20, (j + c[qq, 1]) % 20, (k + c[qq, 2]) % 20
            if fl3[kk, jj, ii] != 0:
                exp.append((idx, qq, pidf[ii + 20 * (jj + 20 * kk)]))
    assert len(exp) == len(cell)
    assert np.all(np.array([e[0] for e in exp]) == cell)
    assert np.all(np.array([e[1] for e in exp]) == q)
    assert np.all(np.array([e[2] for e in exp], np.uint32) == pid)
    assert np.any(pid == 0) and np.any(pid == 0xFFFFFFFE) and np.any(pid == 0xFFFFFFFD)


@pytest.mark.parametrize("shape", [0, 1])
def test_periodic_shift_invariance_of_a_moving_body(shape):
    """Moving every body by a whole number of cells along the periodic axes
    shifts the whole evolution: the same body once in the middle of the shear
    cell and once straddling the x and z seams (lever arms, surface
    velocities, uncovered-cell refill and the position wrap all taken across
    the seam) gives rolled copies of the same fields, force and torque.  The
    summation order of the force differs, so agreement is to rounding."""
    lat = shear_lattice(24, 20, 22, 0.8, 0.02)
    shift = np.array([-10, 0, -9])
    t = np.array([0.7, 0.3, -0.5])
    def run(pos):
        p = Particle(pos=tuple(pos), quat=quat_from_axis(t / np.linalg.norm(t)), semi_axes=(6.0, 2.0, 2.0),
                     vel=(0.012, 0.002, -0.006), omega=(0.0, 0.0, 0.004), density=1.5, shape=shape)
        s = oracle.Sim(lat, [p])
        fl0 = s.fields()[2]
        s.step(100)
        return s, fl0
    a, fl0 = run(np.array([11.5, 9.75, 10.25]))
    b, _ = run(np.array([11.5, 9.75, 10.25]) + shift)
    pa, pb = a.particles()[0], b.particles()[0]
    assert ((fl0 == 0) & (a.fields()[2] != 0)).sum() >= 3       # cells covered ...
    assert ((fl0 == 2) & (a.fields()[2] == 0)).sum() >= 3       # ... and uncovered (refilled)
    dims = np.array([24, 20, 22])
    assert np.allclose((pb[:3] - shift) % dims, pa[:3], rtol=0, atol=1e-12)
    assert np.allclose(pb[3:7], pa[3:7], rtol=0, atol=1e-12)
    fa, fb = a.fields(), b.fields()
    roll = lambda x: np.roll(x.reshape(x.shape[:-1] + (22, 20, 24)), (-shift[2], -shift[0]), axis=(-3, -1))
    assert np.array_equal(roll(fb[2]), fa[2].reshape(22, 20, 24))                 # flags
    assert np.allclose(roll(fb[4]), fa[4].reshape(19, 22, 20, 24), rtol=0, atol=1e-13)
    Fa, Ma = a.forces()
    Fb, Mb = b.forces()
    assert np.allclose(Fb, Fa, rtol=0, atol=1e-11 * np.abs(Fa).max())
    assert np.allclose(Mb, Ma, rtol=0, atol=1e-11 * np.abs(Ma).max())


def _scaled(p, s):
    p.semi_axes = tuple(v * s for v in p.semi_axes)
    return p


def test_momentum_bookkeeping_fixed_particle():
    """Collision conserves momentum and streaming only moves it, so the fluid
    momentum changes by minus the momentum handed to walls and particles."""
    lat = shear_lattice(20, 18, 16, 0.8, 0.02)
    rng = SplitMix64(8)
    p = Particle(pos=(9.7, 8.4, 7.6), quat=quat_from_axis(rng.unit_vector()),
                 semi_axes=(5.0, 2.0, 2.0), fixed=1)
    s = oracle.Sim(lat, [p])
    s.step(30)
    c, _, _ = oracle.lattice_tables()
    for _ in range(5):
        P0 = np.einsum("qn,qa->a", s.fields()[4], c)
        s.step(1)
        P1 = np.einsum("qn,qa->a", s.fields()[4], c)
        F, _ = s.forces()
        Fw = s.wall_forces()
        handed = F[0] + Fw[0] + Fw[1]
        assert np.allclose(P1 - P0, -handed, atol=1e-12 * np.abs(Fw).max(), rtol=0)
        assert np.abs(F[0]).max() > 1e-8


def test_force_on_mirrored_configuration():
    """Mirroring the shear cell in z mirrors the force (F_z flips) and the
    torque (a pseudovector: M_x and M_y flip)."""
    def run(t):
        lat = shear_lattice(16, 18, 16, 1.2, 0.02)
        p = Particle(pos=(7.5, 6.3, 7.5), quat=quat_from_axis(t), semi_axes=(5.0, 2.0, 2.0), fixed=1)
        s = oracle.Sim(lat, [p])
        s.step(300)
        return s.forces()
    t = np.array([0.6, 0.48, 0.64])
    F1, M1 = run(t)
    F2, M2 = run(t * np.array([1, 1, -1]))
    sF = np.array([1, 1, -1])
    sM = np.array([-1, -1, 1])
    scale = np.abs(F1).max()
    assert scale > 1e-6
    assert np.allclose(F2[0], sF * F1[0], atol=1e-12 * scale, rtol=0)
    assert np.allclose(M2[0], sM * M1[0], atol=1e-11 * np.abs(M1).max(), rtol=0)


def test_spinning_particle_feels_opposing_torque():
    lat = Lattice(24, 24, 24, tau=0.8, periodic=(1, 1, 1))
    om = np.array([0.0, 0.0, 2e-3])
    p = Particle(pos=(11.5, 11.5, 11.5), quat=quat_from_axis((1, 0, 0)), semi_axes=(7, 2.5, 2.5),
                 omega=tuple(om), density=10.0)
    s = oracle.Sim(lat, [p])
    s.step(1)
    _, M = s.forces()
    assert np.dot(M[0], om) < 0
    s.step(50)
    assert abs(s.particles()[0][12]) < abs(om[2])


def test_refilled_cells_hold_equilibrium_of_surface_velocity():
    """Uncovered cells get f^eq(rho0, u_s) with u_s from the previous state: their
    density is rho0 and their velocity u_s, exactly (equilibrium moments)."""
    lat = Lattice(30, 14, 14, tau=0.8, periodic=(1, 1, 1))
    p = Particle(pos=(10.0, 6.5, 6.5), quat=quat_from_axis((0.8, 0.6, 0.0)), semi_axes=(5.0, 3.0, 3.0),
                 vel=(0.05, 0.0, 0.0), omega=(0.0, 0.0, 0.01), density=50.0)
    s = oracle.Sim(lat, [p])
    seen = 0
    for _ in range(20):
        before = s.particles()[0].copy()
        fl0 = s.fields()[2]
        s.step(1)
        rho, u, fl1, _, _ = s.fields()
        new = np.nonzero((fl0 == 2) & (fl1 == 0))[0]
        for idx in new:
            i, j, k = idx % 30, (idx // 30) % 14, idx // (30 * 14)
            d = np.array([i, j, k], float) - before[0:3]
            for a, n in enumerate((30, 14, 14)):
                d[a] -= n * round(d[a] / n)
            us = before[7:10] + np.cross(before[10:13], d)
            assert rho[idx] == pytest.approx(1.0, abs=1e-15)
            assert np.allclose(u[:, idx], us, atol=1e-16)
            seen += 1
    assert seen > 10


def test_rigid_body_constant_force():
    rec = oracle.particle_records([Particle(pos=(5.0, 5.0, 5.0), quat=(1, 0, 0, 0),
                                            semi_axes=(3.0, 1.0, 1.0), density=2.0)])[0]
    m, _ = oracle.mass_inertia(rec)
    L = np.zeros(3)
    F = np.array([1e-3, -2e-3, 5e-4])
    x0 = rec[0:3].copy()
    n = 100
    for _ in range(n):
        oracle.rigid_body_step(rec, L, F, np.zeros(3))
    assert np.allclose(rec[7:10], n * F / m, rtol=1e-12, atol=0)
    assert np.allclose(rec[0:3], x0 + F / m * n * (n + 1) / 2, rtol=1e-12, atol=0)
    assert np.allclose(rec[3:7], [1, 0, 0, 0], atol=0)


def test_rigid_body_inertia_of_spheroid():
    rec = oracle.particle_records([Particle(pos=(0, 0, 0), quat=(1, 0, 0, 0), semi_axes=(4.0, 1.5, 1.5),
                                            density=3.0)])[0]
    m, I = oracle.mass_inertia(rec)
    assert m == pytest.approx(3.0 * 4 / 3 * math.pi * 4 * 1.5 * 1.5, rel=1e-15)
    # solid-ellipsoid moments: m/5 (b^2 + c^2) etc.
    assert I[0] == pytest.approx(m * (2 * 1.5 ** 2) / 5, rel=1e-15)
    assert I[1] == pytest.approx(m * (4 ** 2 + 1.5 ** 2) / 5, rel=1e-15)


def test_torque_free_symmetric_top_precesses():
    """Torque-free axisymmetric body: L is constant, the symmetry axis keeps
    its angle to L and precesses about L at rate |L| / I_perp."""
    rec = oracle.particle_records([Particle(pos=(0, 0, 0), quat=quat_from_axis((0.6, 0.0, 0.8)),
                                            semi_axes=(4.0, 1.5, 1.5), density=1.0,
                                            omega=(0.0, 0.0, 0.0))])[0]
    m, I = oracle.mass_inertia(rec)
    L0 = np.array([0.0, 0.0, 2e-4 * I[1]])
    L = L0.copy()
    t0 = np.array(axis_from_quat(rec[3:7]))
    n = 2000
    for _ in range(n):
        oracle.rigid_body_step(rec, L, np.zeros(3), np.zeros(3))
    assert np.array_equal(L, L0)
    t = np.array(axis_from_quat(rec[3:7]))
    Lh = L0 / np.linalg.norm(L0)
    assert np.dot(t, Lh) == pytest.approx(np.dot(t0, Lh), abs=1e-4)  # first order: O(n |Omega|^2)
    rate = np.linalg.norm(L0) / I[1]
    phi = rate * n
    R = np.array([[math.cos(phi), -math.sin(phi), 0], [math.sin(phi), math.cos(phi), 0], [0, 0, 1]])
    assert np.allclose(t, R @ t0, atol=2e-3)


def test_stokes_drag_on_periodic_sphere_array():
    """Fixed sphere in a periodic box driven by a body force: at steady state
    the sphere takes all the injected momentum, and the drag matches
    6 pi mu a U K(c) (Hasimoto) within the staircase accuracy."""
    n, a, tau, g = 20, 4.0, 1.5, 2e-6
    lat = Lattice(n, n, n, tau=tau, periodic=(1, 1, 1), body_force=(g, 0, 0))
    p = Particle(pos=(9.5, 9.5, 9.5), quat=(1, 0, 0, 0), semi_axes=(a, a, a), fixed=1)
    s = oracle.Sim(lat, [p])
    s.step(2500)
    rho, u, fl, _, _ = s.fields()
    F, _ = s.forces()
    nfluid = (fl == 0).sum()
    # momentum balance at steady state: drag = injected momentum per step
    assert F[0][0] == pytest.approx(g * nfluid, rel=2e-3)
    nu = cf.lattice_viscosity(tau)
    U = u[0].sum() / lat.ncells                 # superficial velocity
    c = 4 / 3 * math.pi * a ** 3 / lat.ncells
    stokes = 6 * math.pi * nu * a * U * cf.hasimoto_drag_factor(c)
    assert F[0][0] == pytest.approx(stokes, rel=0.10)


def test_rotating_sphere_torque_matches_the_rotlet():
    """A sphere of radius a spinning at Omega in fluid at rest feels the
    Stokes torque -8 pi mu a^3 Omega (Kirchhoff); the periodic images change
    it by O((a/L)^3).  The 32^3 box with a = 6 after 400 steps (several
    viscous times a^2 / nu) gives the closed form within the staircase
    accuracy, and no torque across the spin axis.  The torque's lever arm,
    the cross product and the surface velocity Omega x (x_s - x_C) of the
    bounce-back all enter."""
    n, a, tau, om = 32, 6.0, 0.8, 1e-3
    lat = Lattice(n, n, n, tau=tau, periodic=(1, 1, 1))
    c = (n - 1) / 2
    p = Particle(pos=(c + 0.13, c - 0.21, c + 0.07), quat=(1, 0, 0, 0), semi_axes=(a, a, a),
                 omega=(0.0, 0.0, om), fixed=1)
    s = oracle.Sim(lat, [p], openmp=True, threads=min(8, os.cpu_count() or 1))
    s.step(400)
    _, M = s.forces()
    mu = cf.lattice_viscosity(tau)          # rho0 = 1
    T = -8 * math.pi * mu * a ** 3 * om
    assert M[0][2] == pytest.approx(T, rel=0.10)
    assert np.abs(M[0][:2]).max() < 1e-2 * abs(T)


def test_jeffery_period_of_the_oracle_spheroid():
    """Jeffery (1922): a spheroid of aspect ratio r in simple shear turns with
    period T = 2 pi (r + 1/r) / gamma; the angle psi = atan2(r sin phi, cos phi)
    of its axis projected on the flow-gradient plane advances linearly.  The
    32^3 case (spheroid 8, 2, 2, walls +-0.01) started from the Couette
    profile, over 6,000 steps (15 % of a period): the fitted period lies
    within 10 % of the closed form (walls 0.53 body lengths apart, Re ~ 0.03)."""
    w = small_shear(seed=1)
    lat, p = w.lattices[0], w.particles[0]
    r = p.semi_axes[0] / p.semi_axes[1]
    gamma = abs(lat.wall_u_hi[0] - lat.wall_u_lo[0]) / (lat.ny - 2.0)
    T = cf.jeffery_period(r, gamma)
    o = oracle.Sim(lat, [p], openmp=True, threads=min(8, os.cpu_count() or 1))
    # Couette profile between the half-way walls, as equilibrium populations
    y = np.arange(lat.ny, dtype=float)
    ux = lat.wall_u_lo[0] + (lat.wall_u_hi[0] - lat.wall_u_lo[0]) * (y - 0.5) / (lat.ny - 2.0)
    feq_y = np.stack([oracle.equilibrium(lat.rho0, (u, 0.0, 0.0), lat.rho0) for u in ux], axis=1)
    n = lat.nx * lat.ny * lat.nz
    o.set_pdfs(np.ascontiguousarray(feq_y[:, (np.arange(n) // lat.nx) % lat.ny]))
    ts, psi = [], []
    for k in range(25):
        q = o.particles()[0][3:7]
        q = q / np.linalg.norm(q)
        wq, x, yq, z = q
        phi = math.atan2(2 * (x * yq + wq * z), 1 - 2 * (yq * yq + z * z))  # body x axis in the x-y plane
        psi.append(math.atan2(r * math.sin(phi), math.cos(phi)))
        ts.append(250.0 * k)
        if k < 24:
            o.step(250)
    psi, ts = np.unwrap(psi), np.array(ts)
    sel = ts >= 1200
    slope = np.polyfit(ts[sel], psi[sel], 1)[0]
    assert slope < 0
    assert 0.9 < (2 * math.pi / abs(slope)) / T < 1.1

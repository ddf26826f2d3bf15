"""Pins of the slender-body oracle (Sec. 3, `oracle/sbf.py`).

* The non-local operator Kbar is diagonal on Legendre polynomials with
  eigenvalues -2 sum_{i<=n} 1/i: checked by direct quadrature of Eq. Kbar.
* A single fibre's translational mobility equals Cox's slender-spheroid
  friction coefficients (independent derivation, `oracle/closed_forms.py`),
  which pins the geometry parameter d and the local operator.
* Two fibres far apart: the velocity one induces on the other tends to the
  Stokeslet of its force, S(R) F / (8 pi mu).
* Two identical parallel fibres side by side falling broadside move with
  equal velocities, faster than one alone, without turning.
* Reciprocity: the velocity fibre 1 gets from a force on fibre 2 equals, as a
  matrix, the transpose of the velocity fibre 2 gets from a force on fibre 1.
* The Legendre and quadrature truncations converge.
* Heun's method: a torque-driven fibre turns at the closed-form rate with
  second-order error in the time step.
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import sbf


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_kbar_is_diagonal_on_legendre(n):
    integrate = pytest.importorskip("scipy.integrate")
    c = np.zeros(n + 1)
    c[n] = 1.0
    P = lambda x: np.polynomial.legendre.legval(x, c)  # noqa: E731
    for s in (-0.83, -0.2, 0.37, 0.91):
        val = integrate.quad(lambda t: (P(t) - P(s)) / abs(t - s), -1.0, 1.0, points=[s], limit=200,
                             epsabs=1e-13, epsrel=1e-12)[0]
        assert val == pytest.approx(sbf.kbar_eigenvalue(n) * P(s), abs=1e-9)


@pytest.mark.parametrize("aspect", [8.0, 20.0, 50.0])
def test_single_fibre_translation_matches_cox_spheroid(aspect):
    L, mu = 2.0, 1.3
    r = L / aspect
    f = sbf.Fibres([(0, 0, 0)], [(0.3, -0.5, 0.81)], L / 2, r, mu)
    p = f.p[0]
    Fpar, Fperp = 2.0 * p, np.cross(p, (0, 0, 1.0))
    Fperp *= 1.7 / np.linalg.norm(Fperp)
    g_par, g_perp = cf.cox_coefficients(mu, L, r, shape="spheroid")
    _, v, w = f.solve([Fpar], [(0, 0, 0)])
    assert np.allclose(v[0], Fpar / g_par, rtol=1e-13, atol=0)
    assert np.allclose(w[0], 0.0, atol=1e-15)
    _, v, _ = f.solve([Fperp], [(0, 0, 0)])
    assert np.allclose(v[0], Fperp / g_perp, rtol=1e-13, atol=1e-17)


def test_far_fibre_sees_the_stokeslet():
    mu = 1.0
    R = np.array([0.0, 300.0, 40.0])
    f = sbf.Fibres([(0, 0, 0), R], [(1, 0, 0), (0.2, 0.7, 0.3)], 1.0, 0.1, mu)
    F2 = np.array([0.3, -1.0, 0.5])
    _, v, _ = f.solve([(0, 0, 0), F2], [(0, 0, 0), (0, 0, 0)])
    Rv = -R  # from fibre 2 to fibre 1
    d = np.linalg.norm(Rv)
    S = (np.eye(3) + np.outer(Rv, Rv) / d ** 2) / d
    expected = S @ F2 / (8 * math.pi * mu)
    assert np.allclose(v[0], expected, rtol=1e-3, atol=1e-4 * np.abs(expected).max())


def test_side_by_side_fibres_fall_together():
    mu, L = 1.0, 2.0
    f2 = sbf.Fibres([(0, -0.6, 0), (0, 0.6, 0)], [(1, 0, 0), (1, 0, 0)], L / 2, 0.08, mu)
    f1 = sbf.Fibres([(0, 0, 0)], [(1, 0, 0)], L / 2, 0.08, mu)
    F = np.array([0.0, 0.0, -1.0])
    _, v2, w2 = f2.solve([F, F], [(0, 0, 0), (0, 0, 0)])
    _, v1, _ = f1.solve([F], [(0, 0, 0)])
    assert np.allclose(v2[0], v2[1], rtol=1e-12, atol=1e-15)
    assert np.allclose(w2, 0.0, atol=1e-12)
    assert v2[0][2] < v1[0][2] < 0  # the pair settles faster


def test_reciprocity_of_the_pair_mobility():
    mu = 0.9
    f = sbf.Fibres([(0, 0, 0), (0.7, 2.3, -0.4)], [(1, 0.2, 0), (0.1, 0.4, 1.0)], 1.0, 0.07, mu, n_modes=6,
                   n_quad=40)
    M12 = np.zeros((3, 3))
    M21 = np.zeros((3, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        _, v, _ = f.solve([(0, 0, 0), e], [(0, 0, 0), (0, 0, 0)])
        M12[:, a] = v[0]
        _, v, _ = f.solve([e, (0, 0, 0)], [(0, 0, 0), (0, 0, 0)])
        M21[:, a] = v[1]
    assert np.allclose(M12, M21.T, rtol=1e-12, atol=1e-13 * np.abs(M12).max())


def test_truncations_converge():
    args = ([(0, 0, 0), (0.5, 1.4, 0.2)], [(1, 0, 0.3), (0.3, 1.0, 0.0)], 1.0, 0.06, 1.0)
    F = [(0, 0, -1.0), (0.2, 0, -1.0)]
    Mt = [(0, 0.1, 0), (0, 0, 0)]
    ref = sbf.Fibres(*args, n_modes=8, n_quad=64).solve(F, Mt)
    for nm, nq in ((5, 24), (6, 32)):
        got = sbf.Fibres(*args, n_modes=nm, n_quad=nq).solve(F, Mt)
        for a, b in zip(got[1:], ref[1:]):
            assert np.allclose(a, b, rtol=2e-3, atol=2e-4 * np.abs(b).max())


def test_heun_rotation_is_second_order():
    mu, L, r = 1.0, 2.0, 0.1
    Mz = 0.05
    d = sbf.geometry_parameter(r / L)
    omega = 3 * d * Mz / (2 * math.pi * mu * L ** 3)
    T = 1.0 / omega  # one radian
    errs = []
    for nsteps in (20, 40):
        f = sbf.Fibres([(0, 0, 0)], [(1, 0, 0)], L / 2, r, mu)
        for _ in range(nsteps):
            f.step([(0, 0, 0)], [(0, 0, Mz)], T / nsteps)
        angle = math.atan2(f.p[0][1], f.p[0][0])
        errs.append(abs(angle - omega * T))
    assert errs[1] < errs[0] / 3.0


def test_rotation_rate_against_tirado_as_the_paper_reports():
    """Sec. 5.2: the SBF angular velocities exceed Tirado's (cylinder of the
    full length) by almost 90 % at 1/eps = 4 and by more than 50 % at 14."""
    mu, r = 1e-3, 4e-5
    ratios = {}
    for aspect in (4, 14):
        L = aspect * r
        f = sbf.Fibres([(0, 0, 0)], [(1, 0, 0)], L / 2, r, mu)
        M = np.array([0.0, 0.0, 1e-15])
        _, _, w = f.solve([(0, 0, 0)], [M])
        omega_sbf = np.linalg.norm(w[0])
        omega_tir = M[2] / cf.tirado_coefficients(mu, L, r)[2]
        ratios[aspect] = omega_sbf / omega_tir
    assert 1.80 < ratios[4] < 1.90
    assert 1.50 < ratios[14] < 1.60


# --------------------------------------------------------------------------
# periodic box (the form the paper's tumbling runs use)
# --------------------------------------------------------------------------

def _direct(Lb, xi):
    b = sbf.PeriodicStokeslet.__new__(sbf.PeriodicStokeslet)
    b.Lb, b.xi, b.n_real, b.n_fourier = Lb, xi, 3, 12
    return b


def test_ewald_split_does_not_depend_on_the_splitting_parameter():
    pytest.importorskip("scipy.special")
    R = np.array([[0.13, 0.31, -0.22], [0.0, 0.0, 0.0], [0.4, -0.45, 0.1], [0.02, 0.0, 0.01]])
    ref = _direct(1.0, 3.5).correction_direct(R)
    for xi in (5.0, 7.0):
        assert np.allclose(_direct(1.0, xi).correction_direct(R), ref, rtol=1e-10, atol=1e-11)


def test_periodic_correction_at_the_origin_is_hasimotos():
    """A force in a periodic cubic array moves its point by C(0) F / (8 pi mu)
    relative to free space; Hasimoto's sphere-array drag, F = 6 pi mu a U K with
    K = 1 + 1.7601 c^(1/3) + ..., c = 4/3 pi a^3 / Lb^3, gives
    C(0) = -(8/6) 1.7601 (4 pi / 3)^(1/3) / Lb."""
    pytest.importorskip("scipy.special")
    Lb = 2.5
    C0 = _direct(Lb, 3.0).correction_direct(np.zeros((1, 3)))[0]
    expected = -(8.0 / 6.0) * 1.7601 * (4 * math.pi / 3) ** (1 / 3) / Lb
    assert np.allclose(C0, expected * np.eye(3), rtol=2e-5, atol=1e-9)


def test_reflection_rule_and_interpolation():
    pytest.importorskip("scipy.special")
    box = sbf.PeriodicStokeslet(1.0, n_grid=12)
    rng = np.random.default_rng(3)
    R = rng.uniform(-0.5, 0.5, size=(6, 3))
    direct = box.correction_direct(R)
    for s in ([1, -1, 1], [-1, -1, 1], [-1, 1, -1]):
        s = np.array(s, dtype=float)
        refl = box.correction_direct(R * s)
        assert np.allclose(refl, direct * np.outer(s, s)[None], rtol=1e-10, atol=1e-11)
    interp = box.correction(R)
    assert np.abs(interp - direct).max() < 2e-3 * 3.78


def test_single_fibre_in_a_periodic_box_feels_its_images():
    pytest.importorskip("scipy.special")
    Lb, mu = 40.0, 1.0
    box = sbf.PeriodicStokeslet(Lb, n_grid=12)
    F = np.array([0.0, 0.0, -1.0])
    free = sbf.Fibres([(0, 0, 0)], [(1, 0, 0)], 1.0, 0.1, mu)
    per = sbf.Fibres([(0, 0, 0)], [(1, 0, 0)], 1.0, 0.1, mu, box=box)
    _, vf, _ = free.solve([F], [(0, 0, 0)])
    _, vp, wp = per.solve([F], [(0, 0, 0)])
    C0 = box.correction_direct(np.zeros((1, 3)))[0]
    assert np.allclose(vp[0] - vf[0], C0 @ F / (8 * math.pi * mu), rtol=1e-2)
    assert np.allclose(wp, 0.0, atol=1e-12)


def _tumbling_pair(aspect, dist_dx, box_dx, dx, r_dx, mu, Fz, dt=0.01, t_end=9.0):
    """Two fibres aligned with gravity (z), dist apart in x, in a periodic cube:
    the period (successive times the pair is aligned with gravity again), the
    sedimentation distance per period and the velocity extremes of one fibre."""
    r = r_dx * dx
    L = aspect * r
    box = sbf.PeriodicStokeslet(box_dx * dx, n_grid=24)
    d = dist_dx * dx
    f = sbf.Fibres([(-d / 2, 0, 0), (d / 2, 0, 0)], [(0, 0, 1), (0, 0, 1)], L / 2, r, mu, n_modes=5, n_quad=24,
                   box=box)
    F = [(0, 0, Fz), (0, 0, Fz)]
    Mt = [(0, 0, 0), (0, 0, 0)]
    t, z, ang, vel = [], [], [], []
    for n in range(int(t_end / dt)):
        _, v, _ = f.solve(F, Mt)
        t.append(n * dt)
        z.append(f.x[0][2])
        ang.append(math.atan2(f.p[0][0], f.p[0][2]))
        vel.append(v[0].copy())
        f.step(F, Mt, dt)
    ang = np.unwrap(np.array(ang))
    k = np.floor(ang / math.pi)
    cross = np.nonzero(np.diff(k) != 0)[0]
    a, b = cross[0], cross[1]
    T = t[b] - t[a]
    D = z[b] - z[a]
    V = np.array(vel[a:b])
    return T, D, V


@pytest.mark.parametrize("row", [0, 1])
def test_tumbling_pair_reproduces_the_papers_slender_body_table(row):
    """Sec. 6.4: the slender-body rows of the tumbling-pair table (periodic
    cube of 576 dx, water, r = 4 dx, 1/eps = 12)."""
    pytest.importorskip("scipy.special")
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_sbf_tumbling.json")))
    g = gold["rows"][row]
    Fz = gold["force_z_N"][str(g["inverse_eps"])]
    T, D, V = _tumbling_pair(g["inverse_eps"], g["dist_dx"], g["box_dx"], gold["dx_m"], gold["radius_dx"],
                             gold["mu"], Fz)
    assert abs(V[:, 0]).max() * 1e6 == pytest.approx(g["ux_max_um_s"], rel=0.01)
    assert V[:, 2].min() * 1e3 == pytest.approx(g["uz_min_mm_s"], rel=0.015)
    assert V[:, 2].max() * 1e3 == pytest.approx(g["uz_max_mm_s"], rel=0.015)
    assert D / T * 1e3 == pytest.approx(g["U_mm_s"], rel=0.02)
    assert T == pytest.approx(g["T_s"], rel=0.03)
    assert D * 1e3 == pytest.approx(g["D_mm"], rel=0.04)

"""Closed-form relations of the paper's Sec. 2 and Sec. 5, plus Jeffery's period.

TEST INFRASTRUCTURE ONLY (part of the oracle package).

* Cox's friction coefficients for slender cylinders and spheroids
  (Eq. CapsTheorVelLengthwSidewMotionCox).
* Tirado et al.'s translational and rotational friction coefficients of a
  cylinder with end corrections (Eqs. CapsTheorVelLengthwSidesMotionTirado,
  CapsTheorRotatMotionTirado, EndeffLengthwMotionTirado,
  EndeffCorrSidewMotionTirado, EndeffCorrRotatMotionTirado).
* The linear force/velocity relations U = F / gamma_t, omega = M / gamma_r
  (Eq. translationalAngularVelocitySB, Eq. TranslVelocitySB).
* The lattice time step from the viscosity relation (Eq. kinVisc).
* Jeffery's (1922) tumbling period T = 2 pi (r + 1/r) / shear_rate of a
  prolate spheroid of aspect ratio r in simple shear.
* The particle Reynolds number Re_p = U L / nu (Eq. ParticleReynoldsNr).
"""
from __future__ import annotations

import math


def cox_coefficients(mu: float, L: float, r: float, shape: str = "cylinder"):
    """(gamma_par, gamma_perp) of Cox for a body of length L and radius r."""
    eps = r / L
    if shape == "cylinder":
        c1, c2 = -1.5 + math.log(2.0), -0.5 + math.log(2.0)
    elif shape == "spheroid":
        c1, c2 = -0.5, 0.5
    else:
        raise ValueError(shape)
    g_par = 2.0 * math.pi * mu * L / (math.log(1.0 / eps) + c1)
    g_perp = 4.0 * math.pi * mu * L / (math.log(1.0 / eps) + c2)
    return g_par, g_perp


def tirado_corrections(p: float):
    """End corrections (upsilon_par, upsilon_perp, delta_perp) at p = L/(2r)."""
    up = -0.207 + 0.980 / p - 0.133 / p ** 2
    uq = 0.839 + 0.185 / p + 0.233 / p ** 2
    dq = -0.662 + 0.917 / p - 0.050 / p ** 2
    return up, uq, dq


def tirado_coefficients(mu: float, L: float, r: float):
    """(gamma_par, gamma_perp, gamma_rot) of Tirado et al. for a cylinder of
    length L and radius r."""
    p = L / (2.0 * r)
    up, uq, dq = tirado_corrections(p)
    g_par = 2.0 * math.pi * mu * L / (math.log(p) + up)
    g_perp = 4.0 * math.pi * mu * L / (math.log(p) + uq)
    g_rot = math.pi * mu * L ** 3 / (3.0 * (math.log(p) + dq))
    return g_par, g_perp, g_rot


def lattice_time_step(tau: float, dx: float, nu: float) -> float:
    """dt from nu = (tau - 1/2) c_s^2 dx^2 / dt with c_s^2 = 1/3 (Eq. kinVisc)."""
    return (tau - 0.5) / 3.0 * dx * dx / nu


def lattice_viscosity(tau: float) -> float:
    return (tau - 0.5) / 3.0


def jeffery_period(aspect: float, shear_rate: float) -> float:
    """Jeffery's tumbling period of a prolate spheroid, aspect ratio a/b."""
    return 2.0 * math.pi * (aspect + 1.0 / aspect) / shear_rate


def jeffery_angle(t: float, aspect: float, shear_rate: float, phi0: float = 0.0) -> float:
    """In-plane Jeffery orbit angle: tan(phi) = r tan(2 pi t / T + phi0)."""
    T = jeffery_period(aspect, shear_rate)
    return math.atan(aspect * math.tan(2.0 * math.pi * t / T + phi0))


def reynolds(U: float, L: float, nu: float) -> float:
    return U * L / nu


def couette_profile(y, ny: int, u_lo: float, u_hi: float):
    """Linear profile between half-way walls at y = 0.5 and y = ny - 1.5."""
    H = ny - 2.0
    return u_lo + (u_hi - u_lo) * ((y - 0.5) / H)


def poiseuille_profile(y, ny: int, g: float, nu: float):
    """Parabola between half-way walls at y = 0.5 and y = ny - 1.5 for body
    force density g: u = g / (2 nu) (y - 0.5) (ny - 1.5 - y)."""
    return g / (2.0 * nu) * (y - 0.5) * (ny - 1.5 - y)


def hasimoto_drag_factor(c: float) -> float:
    """Drag enhancement K(c) of a simple cubic array of spheres at volume
    fraction c (Hasimoto 1959, leading terms): F = 6 pi mu a U K."""
    return 1.0 / (1.0 - 1.7601 * c ** (1.0 / 3.0) + c - 1.5593 * c ** 2)

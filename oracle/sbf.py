"""Slender-body formulation (Sec. 3, non-local slender body approximation) of
rigid straight fibres in free space or in a cubic periodic box: plain FP64
oracle.

TEST INFRASTRUCTURE ONLY (part of the oracle package): shares no code with
the GPU library.

Fibre m: centre x_m, unit tangent p_m, half length l_m (length L = 2 l),
radius r_m, slenderness eps = r / L, geometry parameter d = -ln(eps^2 e)
(Eq. SBFGeomParam).  Centre-line points x_m + s p_m, s = l sigma, sigma in
[-1, 1].  The force per unit length on fibre m is expanded in Legendre
polynomials (Eq. force_exp, written here in physical units):

    f_m(sigma) = F_m / (2 l_m) + sum_{n=1..N} b_m^n P_n(sigma),

so that its integral over the fibre is the external force F_m.  Eq. sev_fils,

    8 pi mu (xdot + s pdot) = Lam f + (I + p p^T) Kbar[f] + U_contr,
    Lam = d (I + p p^T) + 2 (I - p p^T),

is projected onto P_n using (i) the orthogonality of the P_n on [-1, 1],
(ii) Kbar[P_n] = lambda_n P_n with lambda_n = -2 sum_{i<=n} 1/i (Kbar is
diagonal under the Legendre polynomials; Kbar of a constant is 0), and
(iii) the torque condition of Eq. extra_cond, M = l^2 (2/3) p x b^1.  With
A_n = Lam + lambda_n (I + p p^T) and the interaction projections
Q_m^j = int U_m(sigma) P_j(sigma) dsigma this gives

    n >= 2:  (2 / (2n + 1)) A_n b_m^n + Q_m^n = 0,
    n = 1:   b_m^1 = beta_m p_m + 3 / (2 l^2) (M_m x p_m),
             (2/3) 2 (d + lambda_1) beta_m + p_m . Q_m^1 = 0,
    xdot_m = Lam F / (8 pi mu L) + Q_m^0 / (16 pi mu),
    pdot_m = 3 d (M x p) / (2 pi mu L^3) + 3 / (16 pi mu l) (I - p p^T) Q_m^1,

the last two being Eqs. xadot and padot.  U_contr (Eq. Ucontr_def) sums over
the other fibres with the free-space Green's function of Eq. Gnonper,
G = S + r^2 / 2 D, S the Stokeslet and D the dipole doublet; its projections
Q are integrated by tensor Gauss-Legendre quadrature in (sigma, sigma')
(the integrand is smooth for separated fibres).  The coefficients solve one
dense linear system (np.linalg.solve); the paper uses GMRES on the same
system.  Time stepping: Heun's explicit second-order method with fixed step,
the tangent renormalised after each step.

Periodic box (Sec. 3, extension to periodic boundary conditions): the
Stokeslet is replaced by its periodic sum with zero mean flow
(PeriodicStokeslet, Ewald split, tabulated and interpolated as the paper
describes), every fibre also interacting with its own images; the doublet
term is kept for the nearest image only.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


def geometry_parameter(eps: float) -> float:
    """d = -ln(eps^2 e) (Eq. SBFGeomParam)."""
    return -math.log(eps * eps * math.e)


def kbar_eigenvalue(n: int) -> float:
    """lambda_n with Kbar[P_n] = lambda_n P_n on [-1, 1]."""
    return -2.0 * sum(1.0 / i for i in range(1, n + 1))


def legendre_values(n_max: int, x: np.ndarray) -> np.ndarray:
    """P_0..P_n_max at the points x: array (n_max + 1, len(x))."""
    out = np.zeros((n_max + 1, len(x)))
    for n in range(n_max + 1):
        c = np.zeros(n + 1)
        c[n] = 1.0
        out[n] = npleg.legval(x, c)
    return out


def green(R: np.ndarray, r: float) -> np.ndarray:
    """G(R) = S(R) + r^2/2 D(R) for an array of separations R (..., 3):
    S = (I + Rh Rh^T)/|R|, D = (I - 3 Rh Rh^T)/|R|^3 (Eq. Gnonper)."""
    dist = np.linalg.norm(R, axis=-1)
    Rh = R / dist[..., None]
    I = np.eye(3)
    outer = Rh[..., :, None] * Rh[..., None, :]
    S = (I + outer) / dist[..., None, None]
    D = (I - 3.0 * outer) / (dist ** 3)[..., None, None]
    return S + 0.5 * r * r * D


class PeriodicStokeslet:
    """Stokeslet of a cubic periodic box of side Lb with zero mean flow (the net
    force balanced by a mean pressure gradient), for the periodic form of
    Sec. 3: G_per(R) = S(R_mi) + C(R_mi), R_mi the minimum image and C the
    smooth periodic correction.

    C comes from an Ewald split with the screening phi(k) = (1 + k^2/(4 xi^2))
    exp(-k^2/(4 xi^2)): in Fourier space 8 pi mu u = (8 pi / k^2)(I - k k^T / k^2)
    F, so the smooth part is the lattice sum over k != 0 of
    (8 pi / (V k^2)) (I - k k^T / k^2) phi(k) cos(k . R), and the real-space part
    is 8 pi [I (1/(4 pi r) - A) + grad grad (-r/(8 pi) - B)] summed over images,
    A and B the inverse transforms of phi/k^2 and phi/k^4 (closed forms below;
    grad grad g = g'' rh rh^T + g'/r (I - rh rh^T) for radial g).  As the paper
    does, C is tabulated once on a uniform grid over [0, Lb/2]^3 and
    interpolated trilinearly, using C(-R) = C(R) and C_ij of a reflected R =
    s_i s_j C_ij(R)."""

    def __init__(self, Lb: float, n_grid: int = 24, xi: float | None = None, n_real: int = 2, n_fourier: int = 8):
        self.Lb = float(Lb)
        self.xi = float(xi) if xi is not None else 2.0 * math.sqrt(math.pi) / self.Lb
        self.n_real, self.n_fourier = int(n_real), int(n_fourier)
        self.h = 0.5 * self.Lb / n_grid
        ax = np.arange(n_grid + 1) * self.h
        X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        self.table = self.correction_direct(pts).reshape(n_grid + 1, n_grid + 1, n_grid + 1, 3, 3)
        self.n_grid = n_grid

    def _radial(self, r):
        xi = self.xi
        e = np.exp(-xi * xi * r * r)
        erf_ = _erf(xi * r)
        A = erf_ / (4 * math.pi * r) + xi * e / (4 * math.pi ** 1.5)
        I1 = (r * r / 2) * erf_ + r * e / (2 * xi * math.sqrt(math.pi)) - erf_ / (4 * xi * xi)
        B1p = -I1 / (4 * math.pi * r * r)
        B1pp = -erf_ / (4 * math.pi * r) - 2 * B1p / r
        hp = (2 * xi / math.sqrt(math.pi)) * e / r - erf_ / r ** 2
        hpp = -(4 * xi ** 3 / math.sqrt(math.pi)) * e - (4 * xi / math.sqrt(math.pi)) * e / r ** 2 + 2 * erf_ / r ** 3
        return A, B1p + hp / (16 * math.pi * xi * xi), B1pp + hpp / (16 * math.pi * xi * xi)

    def _real(self, R):
        """Screened real-space part (..., 3, 3) at separations R (..., 3), R != 0."""
        r = np.linalg.norm(R, axis=-1)
        rh = R / r[..., None]
        A, Bp, Bpp = self._radial(r)
        P = rh[..., :, None] * rh[..., None, :]
        I = np.eye(3)
        gp = -1.0 / (8 * math.pi) - Bp
        ddg = (-Bpp)[..., None, None] * P + (gp / r)[..., None, None] * (I - P)
        return 8 * math.pi * (I * (1.0 / (4 * math.pi * r) - A)[..., None, None] + ddg)

    def correction_direct(self, R):
        """C(R) = G_per(R) - S(R) by the Ewald sums, R (n, 3) within the minimum-image cell."""
        R = np.asarray(R, dtype=float).reshape(-1, 3)
        out = np.zeros((len(R), 3, 3))
        n = self.n_real
        for i in range(-n, n + 1):
            for j in range(-n, n + 1):
                for k in range(-n, n + 1):
                    Ri = R + self.Lb * np.array([i, j, k], dtype=float)
                    if i == j == k == 0:
                        # the image at the origin: screened part minus nothing, with the
                        # unscreened Stokeslet removed -> -(smooth part), finite at R = 0
                        out += self._self_term(Ri)
                    else:
                        out += self._real(Ri)
        V = self.Lb ** 3
        m = self.n_fourier
        I = np.eye(3)
        for i in range(-m, m + 1):
            for j in range(-m, m + 1):
                for k in range(-m, m + 1):
                    if i == j == k == 0:
                        continue
                    kv = 2 * math.pi / self.Lb * np.array([i, j, k], dtype=float)
                    k2 = kv @ kv
                    phi = (1 + k2 / (4 * self.xi ** 2)) * math.exp(-k2 / (4 * self.xi ** 2))
                    if phi < 1e-18:
                        continue
                    T = (8 * math.pi / (V * k2)) * (I - np.outer(kv, kv) / k2) * phi
                    out += np.cos(R @ kv)[:, None, None] * T[None]
        return out

    def _self_term(self, R):
        """Screened real part minus the Stokeslet at the central image, i.e. minus
        the smooth free-space part: -8 pi [I A + grad grad B]; at R = 0 its limit
        -8 pi [A(0) + B''(0)] I = -(4 xi / sqrt(pi)) I, with A(0) = 3 xi / (4 pi^1.5)
        and grad grad B(0) = B''(0) I = -xi / (4 pi^1.5) I (B smooth and radial)."""
        r = np.linalg.norm(R, axis=-1)
        out = np.zeros((len(R), 3, 3))
        small = r < 1e-6 * self.Lb
        if np.any(~small):
            Rs = R[~small]
            rr = r[~small]
            rh = Rs / rr[:, None]
            S = (np.eye(3) + rh[:, :, None] * rh[:, None, :]) / rr[:, None, None]
            out[~small] = self._real(Rs) - S
        if np.any(small):
            # A(0): erf(xi r)/(4 pi r) -> xi/(2 pi^1.5), plus xi/(4 pi^1.5).  B = B1 + h/(16 pi xi^2),
            # h = erf(xi r)/r: from (r^2 B1')' = -r erf(xi r)/(4 pi) and erf(xi r) ~ 2 xi r/sqrt(pi),
            # B1''(0) = -xi/(6 pi^1.5); h = (2 xi/sqrt(pi))(1 - xi^2 r^2/3 + ...), h''(0) = -4 xi^3/(3 sqrt(pi))
            out[small] = -(4.0 * self.xi / math.sqrt(math.pi)) * np.eye(3)
        return out

    def correction(self, R):
        """Interpolated C at minimum-image separations R (..., 3)."""
        R = np.asarray(R, dtype=float)
        shp = R.shape[:-1]
        R = R.reshape(-1, 3)
        s = np.sign(R)
        s[s == 0] = 1.0
        a = np.abs(R) / self.h
        i0 = np.clip(np.floor(a).astype(int), 0, self.n_grid - 1)
        t = a - i0
        out = np.zeros((len(R), 3, 3))
        for dx in (0, 1):
            wx = t[:, 0] if dx else 1 - t[:, 0]
            for dy in (0, 1):
                wy = t[:, 1] if dy else 1 - t[:, 1]
                for dz in (0, 1):
                    wz = t[:, 2] if dz else 1 - t[:, 2]
                    out += (wx * wy * wz)[:, None, None] * self.table[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
        out *= s[:, :, None] * s[:, None, :]
        return out.reshape(shp + (3, 3))

    def minimum_image(self, R):
        return R - self.Lb * np.round(R / self.Lb)


def _erf(x):
    from scipy.special import erf
    return erf(x)


class Fibres:
    """Rigid straight fibres in Stokes flow (Sec. 3): free space, or a cubic
    periodic box (box = PeriodicStokeslet) where every fibre also interacts
    with the periodic images of all fibres, itself included (the periodic
    correction C only for its own images); the doublet term is kept for the
    nearest image only (it decays as |R|^-3)."""

    def __init__(self, centres, tangents, half_lengths, radii, mu: float, n_modes: int = 5, n_quad: int = 24,
                 box: PeriodicStokeslet | None = None):
        self.x = np.array(centres, dtype=float).reshape(-1, 3)
        p = np.array(tangents, dtype=float).reshape(-1, 3)
        self.p = p / np.linalg.norm(p, axis=1)[:, None]
        M = len(self.x)
        self.l = np.broadcast_to(np.asarray(half_lengths, dtype=float), (M,)).copy()
        self.r = np.broadcast_to(np.asarray(radii, dtype=float), (M,)).copy()
        self.mu = float(mu)
        self.N = int(n_modes)
        self.sig, self.wq = npleg.leggauss(int(n_quad))
        self.P = legendre_values(self.N, self.sig)  # (N + 1, q)
        self.box = box

    @property
    def d(self) -> np.ndarray:
        return np.array([geometry_parameter(r / (2.0 * l)) for r, l in zip(self.r, self.l)])

    def theta(self, m: int, k: int) -> np.ndarray:
        """Theta[j, n] = int int G(R_mk(s, s')) P_j(sigma) P_n(sigma') l_k dsigma' dsigma,
        (N + 1, N + 1, 3, 3); R_mk = x_m + l_m sigma p_m - (x_k + l_k sigma' p_k)."""
        pm = self.x[m][None, :] + self.l[m] * self.sig[:, None] * self.p[m][None, :]
        pk = self.x[k][None, :] + self.l[k] * self.sig[:, None] * self.p[k][None, :]
        R = pm[:, None, :] - pk[None, :, :]                  # (q, q', 3)
        if self.box is None:
            G = green(R, self.r[k])                          # (q, q', 3, 3)
        else:
            Rm = self.box.minimum_image(R)
            C = self.box.correction(Rm)
            G = C if k == m else green(Rm, self.r[k]) + C
        wP = self.P * self.wq[None, :]                       # (N + 1, q)
        return np.einsum("jq,nr,qrab->jnab", wP, wP, G) * self.l[k]

    def _lam(self, m: int, n: int) -> np.ndarray:
        """A_n = Lam + lambda_n (I + p p^T) of fibre m (A_0 = Lam)."""
        pp = np.outer(self.p[m], self.p[m])
        I = np.eye(3)
        lam = self.d[m] * (I + pp) + 2.0 * (I - pp)
        return lam + (kbar_eigenvalue(n) if n > 0 else 0.0) * (I + pp)

    def solve(self, F, Mt):
        """Legendre coefficients b[m, n] (n = 1..N, index n - 1) for external
        forces F (M, 3) and torques Mt (M, 3), and the velocities
        (xdot, pdot)."""
        F = np.array(F, dtype=float).reshape(-1, 3)
        Mt = np.array(Mt, dtype=float).reshape(-1, 3)
        Mf, N = len(self.x), self.N
        periodic = self.box is not None
        th = {(m, k): self.theta(m, k) for m in range(Mf) for k in range(Mf) if k != m or periodic}
        # known parts of b^1: 3 / (2 l^2) (M x p)
        bperp = np.array([3.0 / (2.0 * self.l[m] ** 2) * np.cross(Mt[m], self.p[m]) for m in range(Mf)])
        # unknowns per fibre: beta (1), b^2..b^N (3 each)
        nu = 1 + 3 * (N - 1)
        A = np.zeros((Mf * nu, Mf * nu))
        rhs = np.zeros(Mf * nu)

        def b_of(k):
            """Map of fibre k's b^n (n = 0..N; n = 0 stands for F/(2l)) to unknowns:
            b^n = c_n + E_n z_k with z_k the fibre's unknowns."""
            c = np.zeros((N + 1, 3))
            E = np.zeros((N + 1, 3, nu))
            c[0] = F[k] / (2.0 * self.l[k])
            c[1] = bperp[k]
            E[1, :, 0] = self.p[k]
            for n in range(2, N + 1):
                E[n, :, 1 + 3 * (n - 2):1 + 3 * (n - 1)] = np.eye(3)
            return c, E

        maps = [b_of(k) for k in range(Mf)]
        for m in range(Mf):
            rows = slice(m * nu, (m + 1) * nu)
            # Q_m^j = sum_k sum_n Theta[j, n] b_k^n
            Qc = np.zeros((N + 1, 3))
            QE = np.zeros((N + 1, 3, Mf * nu))
            for k in range(Mf):
                if (m, k) not in th:
                    continue
                c, E = maps[k]
                t = th[(m, k)]
                Qc += np.einsum("jnab,nb->ja", t, c)
                QE[:, :, k * nu:(k + 1) * nu] += np.einsum("jnab,nbu->jau", t, E)
            # own terms
            c, E = maps[m]
            own = np.zeros((nu, Mf * nu))
            ownc = np.zeros(nu)
            # n = 1 parallel: (4/3)(d + lambda_1) beta + p . Q^1 = 0
            own[0, m * nu] += (4.0 / 3.0) * (self.d[m] + kbar_eigenvalue(1))
            own[0] += self.p[m] @ QE[1]
            ownc[0] += self.p[m] @ Qc[1]
            for n in range(2, N + 1):
                r3 = slice(1 + 3 * (n - 2), 1 + 3 * (n - 1))
                own[r3, m * nu + 1 + 3 * (n - 2): m * nu + 1 + 3 * (n - 1)] += 2.0 / (2 * n + 1) * self._lam(m, n)
                own[r3] += QE[n]
                ownc[r3] += Qc[n]
            A[rows] = own
            rhs[rows] = -ownc
        z = np.linalg.solve(A, rhs) if Mf * nu else np.zeros(0)
        b = np.zeros((Mf, N, 3))
        xdot = np.zeros((Mf, 3))
        pdot = np.zeros((Mf, 3))
        bfull = []
        for k in range(Mf):
            c, E = maps[k]
            bk = c + E @ z[k * nu:(k + 1) * nu]
            bfull.append(bk)
            b[k] = bk[1:]
        for m in range(Mf):
            Q = np.zeros((N + 1, 3))
            for k in range(Mf):
                if (m, k) in th:
                    Q += np.einsum("jnab,nb->ja", th[(m, k)], bfull[k])
            L = 2.0 * self.l[m]
            pp = np.outer(self.p[m], self.p[m])
            xdot[m] = self._lam(m, 0) @ F[m] / (8.0 * math.pi * self.mu * L) + Q[0] / (16.0 * math.pi * self.mu)
            pdot[m] = (3.0 * self.d[m] * np.cross(Mt[m], self.p[m]) / (2.0 * math.pi * self.mu * L ** 3)
                       + 3.0 / (16.0 * math.pi * self.mu * self.l[m]) * (np.eye(3) - pp) @ Q[1])
        return b, xdot, pdot

    def step(self, F, Mt, dt: float):
        """One Heun step of Eqs. xadot and padot."""
        x0, p0 = self.x.copy(), self.p.copy()
        _, v1, w1 = self.solve(F, Mt)
        self.x = x0 + dt * v1
        self.p = p0 + dt * w1
        self.p /= np.linalg.norm(self.p, axis=1)[:, None]
        _, v2, w2 = self.solve(F, Mt)
        self.x = x0 + 0.5 * dt * (v1 + v2)
        self.p = p0 + 0.5 * dt * (w1 + w2)
        self.p /= np.linalg.norm(self.p, axis=1)[:, None]

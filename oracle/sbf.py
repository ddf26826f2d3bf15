"""Slender-body formulation (Sec. 3, non-local slender body approximation) of
rigid straight fibres in free space: plain FP64 oracle.

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


class Fibres:
    """Rigid straight fibres in unbounded Stokes flow (Sec. 3)."""

    def __init__(self, centres, tangents, half_lengths, radii, mu: float, n_modes: int = 5, n_quad: int = 24):
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

    @property
    def d(self) -> np.ndarray:
        return np.array([geometry_parameter(r / (2.0 * l)) for r, l in zip(self.r, self.l)])

    def theta(self, m: int, k: int) -> np.ndarray:
        """Theta[j, n] = int int G(R_mk(s, s')) P_j(sigma) P_n(sigma') l_k dsigma' dsigma,
        (N + 1, N + 1, 3, 3); R_mk = x_m + l_m sigma p_m - (x_k + l_k sigma' p_k)."""
        pm = self.x[m][None, :] + self.l[m] * self.sig[:, None] * self.p[m][None, :]
        pk = self.x[k][None, :] + self.l[k] * self.sig[:, None] * self.p[k][None, :]
        R = pm[:, None, :] - pk[None, :, :]                  # (q, q', 3)
        G = green(R, self.r[k])                              # (q, q', 3, 3)
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
        th = {(m, k): self.theta(m, k) for m in range(Mf) for k in range(Mf) if k != m}
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
                if k == m:
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
                if k != m:
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

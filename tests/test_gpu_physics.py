"""GPU checks on the 256x128x128 shear workload (spheroid a = 24, b = 3):

* storage precision: FP32, FP16-offset and BF16-offset runs against the FP64
  oracle after 2,000 steps (velocity relative L2 over fluid cells, force and
  torque of one step from the oracle's state);
* Jeffery's orbit: the body axis of the spheroid rotates with the period
  T = 2 pi (r + 1/r) / gamma of a spheroid of aspect ratio r in simple shear
  (Jeffery 1922); the angle psi = atan2(r sin phi, cos phi) of the axis
  projected on the flow-gradient plane advances linearly in time, so T is
  fitted from a partial orbit.  Walls at 38 % of the body length from each
  other and a finite Reynolds number shift T: the check is a band of 10 %.

Both start from the Couette profile of the moving walls (equilibrium
populations), so the shear is developed at the body from the first step.
"""
import numpy as np
import pytest

from lbm_inputs import large_shear

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
              [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=float)


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_06869_gb300 import _build, lbm as L
    _build.build()
    L.load()
    return L


def couette_pdfs(lat):
    """Equilibrium populations (incompressible, rho0) of the Couette profile
    between the half-way walls at y = 0.5 and y = ny - 1.5."""
    ny = lat.ny
    y = np.arange(ny, dtype=float)
    ulo, uhi = lat.wall_u_lo[0], lat.wall_u_hi[0]
    ux_y = ulo + (uhi - ulo) * (y - 0.5) / (ny - 2.0)
    cu = np.outer(C[:, 0], ux_y)                                  # 19 x ny
    feq_y = W[:, None] * lat.rho0 * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * ux_y[None, :] ** 2)
    n = lat.nx * lat.ny * lat.nz
    jj = (np.arange(n) // lat.nx) % lat.ny
    return np.ascontiguousarray(feq_y[:, jj])


def start(L, w, prec):
    sim = L.Simulation(w.lattices, w.particles, prec=prec)
    sim.set_pdfs(couette_pdfs(w.lattices[0]))
    return sim


def particles_from_records(recs, template):
    from lbm_inputs import Particle
    out = []
    for r, t in zip(recs, template):
        out.append(Particle(pos=tuple(r[0:3]), quat=tuple(r[3:7]), vel=tuple(r[7:10]), omega=tuple(r[10:13]),
                            semi_axes=t.semi_axes, density=t.density))
    return out


def test_storage_precision_against_the_oracle(lbm):
    """The precision study of the 256x128x128 workload: FP32, FP16-offset and
    BF16-offset runs against the FP64 oracle (OpenMP over the host cores)
    after 2,000 steps from the same Couette start -- velocity relative L2 over
    fluid cells -- and the per-step force/torque error: one step of each form
    from the oracle's state after 2,000 steps against the oracle's step."""
    import os
    import oracle
    w = large_shear(seed=1)
    lat = w.lattices[0]
    steps = 2000
    o = oracle.Sim(lat, w.particles, openmp=True, threads=os.cpu_count() or 1)
    o.set_pdfs(couette_pdfs(lat))
    o.step(steps)
    _, u0, fl0, _, pdfs0 = o.fields()
    parts = particles_from_records(o.particles(), w.particles)
    o.step(1)
    F0, M0 = o.forces()
    F0, M0 = F0[0], M0[0]
    runs, loads = {}, {}
    for prec in ("f32", "f16", "bf16"):
        s = start(lbm, w, prec)
        s.step(steps)
        _, u, fl, _, _ = s.fields(0, pdfs=False)
        runs[prec] = (u, fl)
        s.close()
        s = lbm.Simulation([lat], parts, prec=prec)
        s.set_pdfs(pdfs0)
        s.step(1)
        F, M = s.forces()
        loads[prec] = (F[0], M[0])
        s.close()
    # The body sits at the centre of a symmetric shear and rotates almost
    # freely: its net force is round-off and its torque nearly zero, so both
    # are measured against the hydrodynamic scales mu gamma a b and
    # mu gamma a^2 b (mu = rho0 (tau - 1/2) / 3).
    a, b = w.particles[0].semi_axes[0], w.particles[0].semi_axes[1]
    mu = lat.rho0 * (lat.tau - 0.5) / 3.0
    gamma = abs(lat.wall_u_hi[0] - lat.wall_u_lo[0]) / (lat.ny - 2.0)
    sF, sM = mu * gamma * a * b, mu * gamma * a * a * b
    # velocity: the stated 1e-2 of the reduced-precision storage forms; FP32
    # (1e-5 in the short parity runs) accumulates round-off differences of
    # the body's trajectory over 2,000 steps; forces and torques as the
    # full-size parity test
    tol = {"f32": (1e-4, 1e-4), "f16": (1e-2, 2e-2), "bf16": (1e-2, 5e-2)}
    report = {}
    for prec in tol:
        u, fl = runs[prec]
        F, M = loads[prec]
        m = (fl0 == 0) & (fl == 0)
        eu = np.linalg.norm(u[:, m] - u0[:, m]) / np.linalg.norm(u0[:, m])
        eF = np.linalg.norm(F - F0) / sF
        eM = np.linalg.norm(M - M0) / sM
        report[prec] = (eu, eF, eM)
    print("storage precision vs the FP64 oracle: velocity rel L2 after 2000 steps, per-step |dF|/(mu g a b), "
          "|dM|/(mu g a^2 b):", {k: tuple(float(f"{x:.3e}") for x in v) for k, v in report.items()})
    for prec, (eu_max, ef_max) in tol.items():
        eu, eF, eM = report[prec]
        assert eu < eu_max and eF < ef_max and eM < ef_max, (prec, eu, eF, eM)


def test_jeffery_period_from_a_partial_orbit(lbm):
    w = large_shear(seed=1)
    lat, part = w.lattices[0], w.particles[0]
    r = part.semi_axes[0] / part.semi_axes[1]
    gamma = abs(lat.wall_u_hi[0] - lat.wall_u_lo[0]) / (lat.ny - 2.0)
    T_jeffery = 2 * np.pi * (r + 1 / r) / gamma
    s = start(lbm, w, "f32")
    every, nsamp = 500, 40
    t, psi = [], []
    for k in range(nsamp + 1):
        p = s.particles()[0]
        q = p[3:7] / np.linalg.norm(p[3:7])
        wq, x, y, z = q
        axis = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + wq * z), 2 * (x * z - wq * y)])  # body x in world
        phi = np.arctan2(axis[1], axis[0])
        psi.append(np.arctan2(r * np.sin(phi), np.cos(phi)))
        t.append(k * every)
        if k < nsamp:
            s.step(every)
    s.close()
    psi = np.unwrap(np.array(psi))
    t = np.array(t, dtype=float)
    # skip the first 2000 steps (the body spins up from rest)
    sel = t >= 2000
    slope = np.polyfit(t[sel], psi[sel], 1)[0]
    T_fit = 2 * np.pi / abs(slope)
    print(f"Jeffery period: fitted {T_fit:.0f} steps over {int(t[-1])} steps, "
          f"closed form {T_jeffery:.0f} (ratio {T_fit / T_jeffery:.3f})")
    assert slope < 0  # clockwise in the x-y plane for u_x = gamma y
    assert 0.9 < T_fit / T_jeffery < 1.1

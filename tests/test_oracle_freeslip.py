"""Pins of the oracle's free-slip walls (Eq. FreeSlipBC: a population leaving
a fluid cell into the wall is reflected, its normal component reversed, and
arrives at the fluid cell beside its source).

* Mirror images: a box with free-slip walls on an axis evolves exactly like
  the periodic box of twice the fluid extent along that axis started from the
  mirror-symmetric state (the mirror planes are the half-way wall planes).
  Checked for walls on y, on x, and on x and y together (edges).
* A uniform flow tangential to free-slip walls is a steady state (no wall
  stress), while the same flow between resting no-slip walls decays.
* Mass is conserved.
"""
import numpy as np
import pytest

import oracle
from lbm_inputs import Lattice

C, W, OPP = oracle.lattice_tables()


def mirror_dir(axis):
    """Index map q -> direction with component `axis` reversed."""
    out = np.zeros(19, int)
    for q in range(19):
        c = C[q].copy()
        c[axis] = -c[axis]
        out[q] = int(np.nonzero((C == c).all(axis=1))[0][0])
    return out


def random_state(shape, seed, mean=(0.0, 0.0, 0.0)):
    """Populations (19, nz, ny, nx) near equilibrium with random velocity."""
    rng = np.random.default_rng(seed)
    u = np.asarray(mean)[:, None, None, None] + 0.01 * rng.standard_normal((3,) + shape)
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    cu = np.einsum("qa,a...->q...", C.astype(float), u)
    uu = (u * u).sum(axis=0)
    f = W[:, None, None, None] * (rho[None] + 3 * cu + 4.5 * cu * cu - 1.5 * uu[None])
    return f + 1e-4 * rng.standard_normal(f.shape)


def run_free_slip_vs_mirror(axes, dims_fluid, steps=12, seed=1):
    """axes: free-slip axes (0 = x, 1 = y, 2 = z); the others are periodic."""
    nfx, nfy, nfz = dims_fluid
    fs = tuple(1 if a in axes else 0 for a in range(3))
    per = tuple(0 if a in axes else 1 for a in range(3))
    # free-slip box: one wall layer on each side of every free-slip axis
    dims = tuple(n + 2 if a in axes else n for a, n in enumerate(dims_fluid))
    lat = Lattice(*dims, tau=0.85, periodic=per, free_slip=fs)
    s = oracle.Sim(lat)
    f_fluid = random_state((nfz, nfy, nfx), seed, mean=(0.01, -0.005, 0.007))
    f = np.repeat(W[:, None, None, None], dims[2], 1).repeat(dims[1], 2).repeat(dims[0], 3).copy()
    sl = tuple(slice(1, -1) if a in axes else slice(None) for a in (2, 1, 0))
    f[(slice(None),) + sl] = f_fluid
    s.set_pdfs(f.reshape(19, -1))
    # periodic box doubled along every free-slip axis, mirror-symmetric
    g = f_fluid
    for a in axes:
        ax = 3 - a  # array axis of lattice axis a in (q, z, y, x)
        g = np.concatenate([g, np.flip(g, axis=ax)[mirror_dir(a)]], axis=ax)
    dims_p = tuple(2 * n if a in axes else n for a, n in enumerate(dims_fluid))
    latp = Lattice(*dims_p, tau=0.85, periodic=(1, 1, 1))
    p = oracle.Sim(latp)
    p.set_pdfs(g.reshape(19, -1))
    s.step(steps)
    p.step(steps)
    fs_out = s.fields()[4].reshape((19,) + dims[::-1])[(slice(None),) + sl]
    pp_out = p.fields()[4].reshape((19,) + dims_p[::-1])[:, :nfz, :nfy, :nfx]
    return fs_out, pp_out


@pytest.mark.parametrize("axes", [(1,), (0,), (0, 1)])
def test_free_slip_equals_mirror_image_periodic_box(axes):
    a, b = run_free_slip_vs_mirror(axes, (7, 6, 5))
    assert np.allclose(a, b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("free_slip,decays", [((0, 1, 0), False), ((0, 0, 0), True)])
def test_tangential_uniform_flow_along_free_slip_walls(free_slip, decays):
    lat = Lattice(8, 10, 6, tau=0.9, periodic=(1, 0, 1), free_slip=free_slip)
    s = oracle.Sim(lat)
    u0 = np.array([0.02, 0.0, -0.01])
    feq = oracle.equilibrium(1.0, u0)
    s.set_pdfs(np.repeat(feq[:, None], lat.ncells, axis=1))
    s.step(30)
    _, u, fl, _, _ = s.fields()
    err = np.abs(u[:, fl == 0] - u0[:, None]).max()
    if decays:
        assert err > 1e-3
    else:
        assert err < 1e-15


def test_mass_conserved_in_free_slip_box():
    lat = Lattice(9, 8, 7, tau=0.7, periodic=(0, 0, 0), free_slip=(1, 1, 1))
    s = oracle.Sim(lat)
    f = random_state((7, 8, 9), 3, mean=(0.01, 0.02, -0.01)).reshape(19, -1)
    s.set_pdfs(f)
    _, _, fl, _, _ = s.fields()
    m0 = f[:, fl == 0].sum()
    s.step(20)
    rho, _, fl, _, _ = s.fields()
    assert abs(rho[fl == 0].sum() - m0) < 1e-12 * m0


def mirrored_body(p, yc):
    """The image of body p in the plane y = const through which yc is its
    mirrored centre: velocity (vx, -vy, vz), angular velocity (a pseudovector)
    (-wx, wy, -wz), and the rotation M R M with M = diag(1, -1, 1), whose
    quaternion is (w, -x, y, -z).  The shapes are symmetric in their own
    axes, so this is the mirrored body."""
    from lbm_inputs import Particle
    w, x, y, z = p.quat
    return Particle(pos=(p.pos[0], yc, p.pos[2]), quat=(w, -x, y, -z), semi_axes=p.semi_axes,
                    vel=(p.vel[0], -p.vel[1], p.vel[2]), omega=(-p.omega[0], p.omega[1], -p.omega[2]),
                    density=p.density, fixed=p.fixed, shape=p.shape)


@pytest.mark.parametrize("fixed,shape", [(1, 0), (0, 0), (1, 1)])
def test_body_beside_a_free_slip_wall_equals_the_mirrored_pair(fixed, shape):
    """A body next to free-slip y walls evolves like the body and its mirror
    image in the periodic box of twice the fluid height: the moving-obstacle
    bounce-back, the free-slip reflection and cells that have links to both
    agree with the mirror construction, fields and force alike.  A fixed body
    (prescribed velocity and spin) must agree to rounding; a free one moves
    under forces whose summation order differs between the body and its image."""
    from lbm_inputs import Particle, quat_from_axis
    nfx, nfy, nfz = 12, 9, 10
    steps = 10
    lat = Lattice(nfx, nfy + 2, nfz, tau=0.8, periodic=(1, 0, 1), free_slip=(0, 1, 0))
    t = np.array([0.2, 0.97, 0.14])
    body = Particle(pos=(5.5, 4.5, 4.75), quat=quat_from_axis(t / np.linalg.norm(t)),
                    semi_axes=(3.0, 1.5, 1.5), vel=(0.01, -0.004, 0.003), omega=(0.002, -0.001, 0.003),
                    density=2.0, fixed=fixed, shape=shape)
    s = oracle.Sim(lat, [body])
    f_fluid = random_state((nfz, nfy, nfx), 5, mean=(0.01, -0.005, 0.007))
    f = np.repeat(W[:, None, None, None], nfz, 1).repeat(nfy + 2, 2).repeat(nfx, 3).copy()
    f[:, :, 1:-1, :] = f_fluid
    s.set_pdfs(f.reshape(19, -1))
    _, _, fl, pid, _ = s.fields()
    fl = fl.reshape(nfz, nfy + 2, nfx)
    solid = (pid.reshape(fl.shape) != 0xFFFFFFFF)
    assert solid[:, 2, :].any() and not solid[:, 1, :].any()   # cells of row y = 1 touch wall and body

    yb = body.pos[1] - 1.0                                     # height in the doubled periodic box
    latp = Lattice(nfx, 2 * nfy, nfz, tau=0.8, periodic=(1, 1, 1))
    b1 = Particle(pos=(body.pos[0], yb, body.pos[2]), quat=body.quat, semi_axes=body.semi_axes,
                  vel=body.vel, omega=body.omega, density=body.density, fixed=fixed, shape=shape)
    p = oracle.Sim(latp, [b1, mirrored_body(b1, 2 * nfy - 1 - yb)])
    g = np.concatenate([f_fluid, np.flip(f_fluid, axis=2)[mirror_dir(1)]], axis=2)
    p.set_pdfs(g.reshape(19, -1))
    _, _, flp, pidp, _ = p.fields()
    pidp = pidp.reshape(nfz, 2 * nfy, nfx)
    assert np.array_equal(pidp[:, :nfy] == 0, solid[:, 1:-1])
    assert np.array_equal(pidp[:, nfy:] == 1, np.flip(solid[:, 1:-1], axis=1))

    s.step(steps)
    p.step(steps)
    tol = 1e-15 if fixed else 1e-12
    _, _, fl, _, fs_out = s.fields()
    fs_out = fs_out.reshape(19, nfz, nfy + 2, nfx)[:, :, 1:-1]
    pp_out = p.fields()[4].reshape(19, nfz, 2 * nfy, nfx)[:, :, :nfy]
    assert np.allclose(fs_out, pp_out, rtol=0, atol=tol)
    Fs, Ms = s.forces()
    Fp, Mp = p.forces()
    assert np.abs(Fs).max() > 1e-4
    assert np.allclose(Fs[0], Fp[0], rtol=0, atol=1e3 * tol * np.abs(Fs).max())
    assert np.allclose(Ms[0], Mp[0], rtol=0, atol=1e3 * tol * np.abs(Ms).max())
    # the image feels the mirrored force and torque
    assert np.allclose(Fp[1], Fp[0] * [1, -1, 1], rtol=0, atol=1e3 * tol * np.abs(Fs).max())
    assert np.allclose(Mp[1], Mp[0] * [-1, 1, -1], rtol=0, atol=1e3 * tol * np.abs(Ms).max())
    if not fixed:
        xs, xp = s.particles()[0, :3], p.particles()[0, :3]
        assert np.allclose(xs - [0, 1, 0], xp, rtol=0, atol=1e-12)
        assert abs(xs[1] - body.pos[1]) > 1e-6                 # the body did move

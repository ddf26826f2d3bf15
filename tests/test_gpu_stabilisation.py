"""Momentum stabilisation (Sec. 4.1) on the GPU: the CUDA path against the
FP64 oracle in a fully periodic box with bodies under constant external
forces (the setting the paper uses it in), and the exact decay of the total
fluid momentum, J_{n+1} = (1 - omega_odd) J_n, in a periodic box without
obstacles.
"""
import numpy as np
import pytest

import oracle
from lbm_inputs import Lattice, Particle, SplitMix64, quat_from_axis, SHAPE_SPHEROCYLINDER

pytestmark = pytest.mark.gpu

TOL_U = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_06869_gb300 import _build, lbm as L
    _build.build()
    L.load()
    return L


def random_state(lat, seed, mean):
    rng = np.random.default_rng(seed)
    c, w, _ = oracle.lattice_tables()
    n = lat.ncells
    u = np.asarray(mean)[:, None] + 0.005 * rng.standard_normal((3, n))
    rho = 1.0 + 0.005 * rng.standard_normal(n)
    cu = c @ u
    uu = (u * u).sum(axis=0)
    return w[:, None] * (rho[None, :] + 3 * cu + 4.5 * cu * cu - 1.5 * uu[None, :])


def rel_l2(a, b, mask):
    a, b = a[..., mask], b[..., mask]
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_stabilised_periodic_box_with_forced_bodies(lbm, prec):
    lat = Lattice(26, 22, 24, tau=0.9, periodic=(1, 1, 1))
    rng = SplitMix64(31)
    ps = [Particle(pos=(8.3, 10.6, 11.9), quat=quat_from_axis(rng.unit_vector()), semi_axes=(6.0, 2.3, 2.3),
                   shape=SHAPE_SPHEROCYLINDER, density=1.5, ext_force=(0.0, 0.0, -0.3)),
          Particle(pos=(19.2, 11.1, 12.4), quat=quat_from_axis(rng.unit_vector()), semi_axes=(4.5, 2.2, 2.0),
                   density=1.5, ext_force=(0.0, 0.0, -0.2), ext_torque=(0.0, 1.0, 0.0))]
    g = lbm.Simulation(lat, ps, prec=prec)
    o = oracle.Sim(lat, ps)
    f0 = random_state(lat, 5, mean=(0.004, -0.002, 0.003))
    _, _, fl, _, _ = o.fields()
    f0[:, fl != 0] = oracle.lattice_tables()[1][:, None]  # rest populations in the bodies
    g.set_pdfs(f0)
    o.set_pdfs(f0)
    g.set_momentum_stabilisation(True)
    o.set_momentum_stabilisation(True)
    for c in (1, 2, 5, 12, 20):
        g.step(c)
        o.step(c)
        _, ug, fg, pg, _ = g.fields()
        _, uo, fo, po, _ = o.fields()
        assert np.array_equal(fg, fo) and np.array_equal(pg, po)
        e = rel_l2(ug, uo, fo == 0)
        assert e <= TOL_U[prec], f"velocity rel L2 {e:.3e}"
    pgr, por = g.particles(), o.particles()
    assert np.allclose(pgr[:, 0:13], por[:, 0:13], rtol=1e-9 if prec == "f64" else 1e-4, atol=1e-12)
    # the stabilised fluid does not drift with the sinking bodies
    mean_u = uo[:, fo == 0].mean(axis=1)
    assert abs(mean_u[2]) < 0.2 * abs(por[:, 9]).max()


@pytest.mark.parametrize("prec,rtol", [("f64", 1e-11), ("f32", 1e-4)])
def test_total_momentum_decays_exactly(lbm, prec, rtol):
    tau = 1.3
    lat = Lattice(40, 36, 33, tau=tau, periodic=(1, 1, 1))
    g = lbm.Simulation(lat, [], prec=prec)
    g.set_pdfs(random_state(lat, 6, mean=(0.01, -0.006, 0.008)))
    g.set_momentum_stabilisation(True)
    oo = oracle.omega_odd(tau, lat.magic)

    def J():
        return g.fields()[1].sum(axis=1)

    j = J()
    for n in (1, 1, 2, 3):
        g.step(n)
        jn = J()
        assert np.allclose(jn, (1 - oo) ** n * j, rtol=rtol, atol=rtol * np.abs(j).max()), (jn, j)
        j = jn


def test_batch_rejects_stabilisation(lbm):
    lats = [Lattice(10, 10, 10, periodic=(1, 1, 1)), Lattice(12, 10, 10, periodic=(1, 1, 1))]
    g = lbm.Simulation(lats, [])
    with pytest.raises(lbm.LBMError):
        g.set_momentum_stabilisation(True)

"""Free-slip walls (Eq. FreeSlipBC) on the GPU against the FP64 oracle: a
channel with free-slip y walls, a closed free-slip box (edges and corners),
free-slip walls meeting no-slip walls, a moving body in a free-slip box, every
sweep variant, and the export/import of the AA state at both parities."""
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


def random_state(lat, seed, mean=(0.01, -0.004, 0.006)):
    rng = np.random.default_rng(seed)
    c, w, _ = oracle.lattice_tables()
    n = lat.ncells
    u = np.asarray(mean)[:, None] + 0.01 * rng.standard_normal((3, n))
    rho = 1.0 + 0.01 * rng.standard_normal(n)
    cu = c @ u
    uu = (u * u).sum(axis=0)
    return w[:, None] * (rho[None, :] + 3 * cu + 4.5 * cu * cu - 1.5 * uu[None, :])


def rel_l2(a, b, mask):
    a, b = a[..., mask], b[..., mask]
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def run_and_compare(lbm, lat, parts, prec, chunks=(1, 2, 5, 12), launch=None, split=False, seed=1):
    g = lbm.Simulation(lat, parts, prec=prec)
    o = oracle.Sim(lat, parts)
    if launch is not None:
        lbm.lbm_set_launch(g.h, launch, 0)
    if split:
        lbm.lbm_set_sweep_split(g.h, True)
    f0 = random_state(lat, seed)
    _, _, fl, _, _ = o.fields()
    f0[:, fl != 0] = oracle.lattice_tables()[1][:, None]
    g.set_pdfs(f0)
    o.set_pdfs(f0)
    for c in chunks:
        g.step(c)
        o.step(c)
        _, ug, fg, pg, dg = g.fields()
        _, uo, fo, po, do_ = o.fields()
        assert np.array_equal(fg, fo) and np.array_equal(pg, po)
        e = rel_l2(ug, uo, fo == 0)
        assert e <= TOL_U[prec], f"after {c}: velocity rel L2 {e:.3e}"
        ef = rel_l2(dg, do_, fo == 0)
        assert ef <= 10 * TOL_U[prec], f"after {c}: populations rel L2 {ef:.3e}"
    return g, o


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_free_slip_channel(lbm, prec):
    lat = Lattice(20, 14, 12, tau=0.8, periodic=(1, 0, 1), free_slip=(0, 1, 0))
    run_and_compare(lbm, lat, [], prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_closed_free_slip_box(lbm, prec):
    lat = Lattice(17, 13, 11, tau=0.7, periodic=(0, 0, 0), free_slip=(1, 1, 1))
    run_and_compare(lbm, lat, [], prec)


def test_free_slip_meets_no_slip(lbm):
    # free-slip y walls, resting no-slip x walls, periodic z: the x-y edges bounce back
    lat = Lattice(15, 12, 10, tau=0.9, periodic=(0, 0, 1), free_slip=(0, 1, 0))
    run_and_compare(lbm, lat, [], "f64")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_body_in_free_slip_box(lbm, prec):
    lat = Lattice(30, 26, 24, tau=0.8, periodic=(0, 0, 0), free_slip=(1, 1, 1))
    rng = SplitMix64(41)
    p = Particle(pos=(14.6, 12.7, 11.9), quat=quat_from_axis(rng.unit_vector()), semi_axes=(6.0, 2.4, 2.4),
                 shape=SHAPE_SPHEROCYLINDER, density=1.5, ext_force=(0.0, 0.0, -0.3), omega=(0.0, 0.01, 0.0))
    g, o = run_and_compare(lbm, lat, [p], prec, chunks=(1, 2, 5, 12, 20))
    assert np.allclose(g.particles()[:, 0:13], o.particles()[:, 0:13], rtol=1e-9 if prec == "f64" else 1e-4,
                       atol=1e-12)


@pytest.mark.parametrize("launch,split", [(0, False), (-1, False), (128, True), (256, False)])
def test_free_slip_every_sweep_variant(lbm, launch, split):
    lat = Lattice(33, 20, 18, tau=0.8, periodic=(0, 0, 0), free_slip=(1, 1, 1))
    p = Particle(pos=(16.2, 9.7, 8.9), quat=quat_from_axis((0.3, 0.5, 0.81)), semi_axes=(5.0, 2.2, 2.0),
                 density=2.0, vel=(0.01, 0.0, 0.005))
    run_and_compare(lbm, lat, [p], "f32", launch=launch, split=split, chunks=(1, 4, 9))


@pytest.mark.parametrize("steps", [0, 1])
def test_state_export_import_round_trip(lbm, steps):
    lat = Lattice(12, 10, 9, tau=0.8, periodic=(0, 0, 0), free_slip=(1, 1, 1))
    g = lbm.Simulation(lat, [], prec="f64")
    g.step(steps)
    f = random_state(lat, 7)
    _, _, fl, _, _ = g.fields()
    f[:, fl != 0] = oracle.lattice_tables()[1][:, None]
    g.set_pdfs(f)
    d = g.fields()[4]
    assert np.abs(d[:, fl == 0] - f[:, fl == 0]).max() <= 1e-16


def test_body_next_to_free_slip_wall_rejected(lbm):
    lat = Lattice(20, 20, 20, periodic=(1, 0, 1), free_slip=(0, 1, 0))
    with pytest.raises(lbm.LBMError):
        lbm.Simulation(lat, [Particle(pos=(10.0, 3.8, 10.0), quat=(1, 0, 0, 0), semi_axes=(2.5, 2.5, 2.5))])
    with pytest.raises(lbm.LBMError):
        lbm.Simulation(Lattice(20, 20, 20, periodic=(1, 1, 1), free_slip=(0, 1, 0)), [])

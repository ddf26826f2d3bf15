"""GPU parity: the CUDA library (through its C interface) against the FP64 CPU
oracle on the same seeded inputs.

Tolerances: flags, particle-id maps and link lists bit-exact; velocity
relative L2 over fluid cells 1e-12 (FP64 storage), 1e-5 (FP32), 1e-2
(FP16/BF16 offsets); forces and torques as stated per test.
"""
import numpy as np
import pytest

import oracle
from lbm_inputs import (Lattice, Particle, SplitMix64, quat_from_axis, shear_lattice, small_shear,
                        batched_shear, DENSITY)

pytestmark = pytest.mark.gpu

TOL_U = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-2, "bf16": 1e-2}


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_06869_gb300 import _build, lbm as L
    _build.build()
    L.load()
    return L


def force_close(Fg, Mg, Fo, Mo, semi_max, tol):
    """Force and torque agree to tol relative to the load scale of the body:
    |M| for torques and max(|F|, |M| / a) for forces (a centred body in
    symmetric shear has a force that is pure round-off)."""
    sM = max(np.abs(Mo).max(), 1e-300)
    sF = max(np.abs(Fo).max(), sM / semi_max)
    eF = np.abs(Fg - Fo).max() / sF
    eM = np.abs(Mg - Mo).max() / sM
    assert eF <= tol and eM <= tol, f"force err {eF:.3e}, torque err {eM:.3e} (tol {tol:.1e})"
    return eF, eM


def rel_l2(a, b, mask=None):
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def run_pair(L, lat, parts, steps, prec, chunks=(None,)):
    g = L.Simulation(lat, parts, prec=prec)
    o = oracle.Sim(lat, parts)
    for c in chunks:
        n = steps if c is None else c
        g.step(n)
        o.step(n)
    return g, o


def compare_state(g, o, prec, cell=0, check_pdfs=True, tol_u=None, pid_offset=0):
    rg, ug, fg, pg, dg = g.fields(cell)
    ro, uo, fo, po, do_ = o.fields()
    if pid_offset:
        # batch: particle ids are global indices, the oracle numbers its own from 0
        part = pg < 0xFFFFFFFC
        pg = pg.copy()
        pg[part] -= np.uint32(pid_offset)
    assert np.array_equal(fg, fo), f"flags differ at {np.nonzero(fg != fo)[0][:10]}"
    assert np.array_equal(pg, po), "particle-id maps differ"
    fluid = fo == 0
    tol = tol_u if tol_u is not None else TOL_U[prec]
    e_u = rel_l2(ug, uo, fluid)
    assert e_u <= tol, f"velocity rel L2 {e_u:.3e} > {tol:.1e}"
    if check_pdfs:
        e_f = rel_l2(dg - oracle_weights()[:, None], do_ - oracle_weights()[:, None], fluid)
        assert e_f <= max(10 * tol, 1e-11), f"population-offset rel L2 {e_f:.3e}"
    return e_u


_W = None


def oracle_weights():
    global _W
    if _W is None:
        _W = oracle.lattice_tables()[1]
    return _W


# --------------------------------------------------------------------------
# fluid only
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_couette_no_particle(lbm, prec):
    lat = shear_lattice(19, 14, 11, 0.8, 0.02)
    g, o = run_pair(lbm, lat, [], 150, prec)
    compare_state(g, o, prec)
    Fw_g, Fw_o = g.wall_forces(), o.wall_forces()
    scale = np.abs(Fw_o).max()
    assert np.allclose(Fw_g, Fw_o, rtol=TOL_U[prec] * 10, atol=TOL_U[prec] * 10 * scale)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fully_periodic_body_force_and_odd_step_counts(lbm, prec):
    lat = Lattice(13, 9, 7, tau=0.7, periodic=(1, 1, 1), body_force=(1e-4, -2e-5, 3e-5))
    g, o = run_pair(lbm, lat, [], 0, prec, chunks=(1, 2, 7, 3))
    compare_state(g, o, prec)


def test_set_pdfs_round_trip_both_parities(lbm):
    lat = shear_lattice(12, 10, 9, 0.9, 0.02)
    rng = np.random.default_rng(3)
    p = Particle(pos=(5.3, 4.6, 4.1), quat=quat_from_axis((0.6, 0.8, 0.0)), semi_axes=(3.0, 1.8, 1.8))
    g = lbm.Simulation(lat, [p], prec="f64")
    for extra in (0, 1):
        g.step(extra)
        _, _, fl, _, d = g.fields()
        d2 = d + np.where(fl == 0, 1e-4 * rng.standard_normal(d.shape), 0.0)
        g.set_pdfs(d2)
        _, _, _, _, d3 = g.fields()
        assert np.abs(d3 - d2).max() <= 1e-16


# --------------------------------------------------------------------------
# with particles
# --------------------------------------------------------------------------

def test_initial_mapping_and_links_bit_exact(lbm):
    w = small_shear(seed=7)
    g = lbm.Simulation(w.lattices[0], w.particles, prec="f64")
    o = oracle.Sim(w.lattices[0], w.particles)
    _, _, fg, pg, _ = g.fields()
    _, _, fo, po, _ = o.fields()
    assert np.array_equal(fg, fo) and np.array_equal(pg, po)
    for a, b in zip(g.links(), o.links()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_small_shear_spheroid_200_steps(lbm, prec):
    """32^3 Couette cell with the (8,2,2) spheroid, 200 steps (the FP64
    oracle-size workload), in every storage form."""
    w = small_shear(seed=1)
    g, o = run_pair(lbm, w.lattices[0], w.particles, w.steps, prec)
    compare_state(g, o, prec)
    for a, b in zip(g.links(), o.links()):
        assert np.array_equal(a, b)
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    tolF = {"f64": 1e-9, "f32": 1e-4, "f16": 0.05, "bf16": 0.1}[prec]
    force_close(Fg, Mg, Fo, Mo, 8.0, tolF)
    pg, po = g.particles(), o.particles()
    assert np.allclose(pg[:, 0:3], po[:, 0:3], atol=1e-9 if prec == "f64" else 1e-5)
    assert np.allclose(pg[:, 10:13], po[:, 10:13], rtol=1e-6 if prec == "f64" else 0.05, atol=1e-9)


@pytest.mark.parametrize("chunks", [(1,), (2,), (1, 1, 1), (5, 4)])
def test_moving_particle_remap_every_parity(lbm, chunks):
    """A body driven through the lattice uncovers and covers cells every step;
    the re-mapping must follow the AA layout at both parities."""
    lat = Lattice(26, 15, 13, tau=0.75, periodic=(1, 0, 1), wall_u_lo=(-0.01, 0, 0),
                  wall_u_hi=(0.01, 0, 0))
    rng = SplitMix64(11)
    ps = [Particle(pos=(24.1, 7.2, 6.3), quat=quat_from_axis(rng.unit_vector()), semi_axes=(4.0, 2.2, 1.9),
                   vel=(0.07, 0.01, -0.02), omega=(0.0, 0.01, 0.02), density=40.0),
          Particle(pos=(8.4, 7.6, 1.2), quat=quat_from_axis(rng.unit_vector()), semi_axes=(3.5, 2.0, 2.0),
                   vel=(-0.05, 0.0, 0.06), omega=(0.03, 0.0, 0.0), density=40.0)]
    g = lbm.Simulation(lat, ps, prec="f64")
    o = oracle.Sim(lat, ps)
    for c in chunks * 3:
        g.step(c)
        o.step(c)
        compare_state(g, o, "f64")
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    force_close(Fg, Mg, Fo, Mo, 4.0, 1e-9)


def test_overlapping_particles_lowest_index_owns(lbm):
    lat = Lattice(20, 16, 16, periodic=(1, 1, 1))
    ps = [Particle(pos=(10.0, 8.0, 8.0), quat=(1, 0, 0, 0), semi_axes=(5.0, 3.0, 3.0), vel=(0.03, 0, 0),
                   density=30.0),
          Particle(pos=(13.0, 8.5, 7.5), quat=quat_from_axis((0, 1, 0)), semi_axes=(5.0, 2.5, 2.5),
                   density=30.0)]
    g, o = run_pair(lbm, lat, ps, 9, "f64")
    compare_state(g, o, "f64")


def test_fixed_particle_and_external_load(lbm):
    lat = shear_lattice(22, 18, 16, 1.0, 0.02)
    ps = [Particle(pos=(10.5, 8.2, 7.7), quat=quat_from_axis((0.48, 0.6, 0.64)), semi_axes=(5.0, 2.0, 2.0),
                   fixed=1),
          Particle(pos=(3.2, 12.5, 12.0), quat=(1, 0, 0, 0), semi_axes=(2.5, 2.5, 2.5),
                   ext_force=(1e-3, 0, 0), ext_torque=(0, 0, 2e-3), density=5.0)]
    g, o = run_pair(lbm, lat, ps, 40, "f64")
    compare_state(g, o, "f64")
    assert np.allclose(g.particles(), o.particles(), rtol=1e-10, atol=1e-12)


def test_ragged_lattice_many_tiles(lbm):
    """Sizes that are not multiples of any block, several tiles, a ragged tail."""
    lat = shear_lattice(37, 23, 19, 0.65, 0.015)
    rng = SplitMix64(5)
    ps = [Particle(pos=(18.1, 11.3, 9.2), quat=quat_from_axis(rng.unit_vector()), semi_axes=(7.0, 3.0, 2.5))]
    g, o = run_pair(lbm, lat, ps, 30, "f32")
    compare_state(g, o, "f32")


def test_minimum_lattice(lbm):
    lat = shear_lattice(3, 3, 3, 0.8, 0.01)
    g, o = run_pair(lbm, lat, [], 5, "f64")
    compare_state(g, o, "f64")


@pytest.mark.parametrize("block", [0, -1, 128, 256])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_every_sweep_variant(lbm, block, prec):
    """Ring (block 0), bulk-copy staged (block -1) and direct sweeps on a
    lattice periodic in all directions (odd steps wrap on every face) with a
    moving body."""
    lat = Lattice(21, 18, 17, tau=0.7, periodic=(1, 1, 1), body_force=(2e-5, 0, 0))
    rng = SplitMix64(17)
    ps = [Particle(pos=(1.5, 9.2, 16.1), quat=quat_from_axis(rng.unit_vector()), semi_axes=(5.0, 2.5, 2.0),
                   vel=(0.02, -0.01, 0.03), omega=(0.0, 0.0, 0.01), density=20.0)]
    g = lbm.Simulation(lat, ps, prec=prec)
    lbm.lbm_set_launch(g.h, block, 0)
    o = oracle.Sim(lat, ps)
    for c in (1, 4, 3):
        g.step(c)
        o.step(c)
        compare_state(g, o, prec)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("block", [128, 256])
def test_split_sweep_matches_oracle(lbm, block, prec):
    """Split direct sweep (near-obstacle cells compacted into a list and
    updated by a kernel of their own): moving walls, three bodies, one of them
    touching another's neighbourhood, every parity."""
    lat = shear_lattice(40, 30, 26, 0.75, 0.015)
    rng = SplitMix64(23)
    ps = [Particle(pos=(12.0, 14.5, 12.5), quat=quat_from_axis(rng.unit_vector()), semi_axes=(7.0, 2.5, 2.5),
                   vel=(0.01, 0.0, -0.005), omega=(0.0, 0.004, 0.002), density=4.0),
          Particle(pos=(27.5, 13.0, 13.0), quat=quat_from_axis(rng.unit_vector()), semi_axes=(5.0, 2.0, 2.0),
                   vel=(-0.01, 0.002, 0.0), density=4.0),
          Particle(pos=(20.0, 21.5, 6.0), quat=quat_from_axis(rng.unit_vector()), semi_axes=(4.0, 2.0, 2.0),
                   omega=(0.01, 0.0, 0.0), density=4.0)]
    g = lbm.Simulation(lat, ps, prec=prec)
    lbm.lbm_set_launch(g.h, block, 0)
    lbm.lbm_set_sweep_split(g.h, True)
    assert lbm.lbm_get_info(g.h).sweep_split == 1
    o = oracle.Sim(lat, ps)
    for c in (1, 4, 3, 12):
        g.step(c)
        o.step(c)
        compare_state(g, o, prec)
    Fg, Mg = g.forces()
    Fo, Mo = o.forces()
    for i in range(len(ps)):
        force_close(Fg[i], Mg[i], Fo[i], Mo[i], max(ps[i].semi_axes), {"f64": 1e-9, "f32": 1e-4, "f16": 5e-2}[prec])


def test_split_sweep_batched(lbm):
    w = batched_shear(seed=7, ncell=3, steps=7)
    g = lbm.Simulation(w.lattices, w.particles, prec="f32")
    lbm.lbm_set_sweep_split(g.h, True)
    g.step(7)
    for c in range(3):
        p = w.particles[c]
        o = oracle.Sim(w.lattices[c], [Particle(**{**p.__dict__, "cell": 0})])
        o.step(7)
        compare_state(g, o, "f32", cell=c, pid_offset=c)


def test_graph_replay_matches_eager(lbm):
    w = small_shear(seed=2, n=24, steps=40)
    a = lbm.Simulation(w.lattices[0], w.particles, prec="f64")
    b = lbm.Simulation(w.lattices[0], w.particles, prec="f64")
    lbm.lbm_set_graphs(b.h, False)
    a.step(40)
    for _ in range(40):
        b.step(1)
    ra, ua, fa, pa, _ = a.fields()
    rb, ub, fb, pb, _ = b.fields()
    assert np.array_equal(fa, fb) and np.array_equal(pa, pb)
    assert rel_l2(ua, ub, fa == 0) < 1e-13


def test_single_step_graphs_match_eager(lbm):
    """Steps taken one call at a time replay the one-step graph of their
    parity; the state equals eager stepping and multi-step graph replay."""
    w = small_shear(seed=4, n=24, steps=21)
    sims = [lbm.Simulation(w.lattices[0], w.particles, prec="f64") for _ in range(3)]
    lbm.lbm_set_graphs(sims[2].h, False)
    for _ in range(21):
        sims[0].step(1)
    sims[1].step(3)
    sims[1].step(18)
    for _ in range(21):
        sims[2].step(1)
    ref = sims[2].fields()
    for s in sims[:2]:
        r, u, f, p, _ = s.fields()
        assert np.array_equal(f, ref[2]) and np.array_equal(p, ref[3])
        assert rel_l2(u, ref[1], ref[2] == 0) < 1e-13
    n1 = lbm.lbm_get_launch_count(sims[0].h)
    assert n1 == lbm.lbm_get_launch_count(sims[2].h)


def test_autotune_keeps_state(lbm):
    lat = shear_lattice(40, 20, 18, 0.8, 0.02)
    g = lbm.Simulation(lat, [], prec="f32")
    g.step(5)
    before = g.fields()
    blk, grd = lbm.lbm_autotune(g.h)
    assert blk in (0, -1, 128, 256) and grd > 0
    after = g.fields()
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    o = oracle.Sim(lat)
    o.step(5)
    g.step(7)
    o.step(7)
    compare_state(g, o, "f32")


# --------------------------------------------------------------------------
# batched lattices
# --------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_of_uneven_lattices(lbm, prec):
    """Independent lattices of different sizes, tau and wall speeds, one
    spheroid each, advanced by one sweep launch per step."""
    rng = SplitMix64(21)
    lats, parts = [], []
    for c, (nx, ny, nz) in enumerate([(20, 16, 17), (25, 18, 14), (17, 21, 19), (30, 15, 16)]):
        tau = 0.6 + 0.6 * rng.uniform()
        uw = 0.005 + 0.025 * rng.uniform()
        lat = shear_lattice(nx, ny, nz, tau, uw)
        b = 1.5 + rng.uniform()
        p = Particle(pos=((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2), quat=quat_from_axis(rng.unit_vector()),
                     semi_axes=(2.5 * b, b, b), cell=c, density=DENSITY)
        lats.append(lat)
        parts.append(p)
    g = lbm.Simulation(lats, parts, prec=prec)
    g.step(60)
    Fg, Mg = g.forces()
    for c, lat in enumerate(lats):
        p = parts[c]
        o = oracle.Sim(lat, [Particle(**{**p.__dict__, "cell": 0})])
        o.step(60)
        compare_state(g, o, prec, cell=c, pid_offset=c)
        Fo, Mo = o.forces()
        force_close(Fg[c:c + 1], Mg[c:c + 1], Fo, Mo, 2.5 * 2.5, 1e-9 if prec == "f64" else 1e-3)


def test_batched_workload_generator_and_first_steps(lbm):
    """The 512-cell batched workload generator: a subset runs and matches the
    oracle cell by cell."""
    w = batched_shear(seed=3, ncell=6, steps=10)
    g = lbm.Simulation(w.lattices, w.particles, prec="f32")
    g.step(10)
    for c in (0, 5):
        p = w.particles[c]
        o = oracle.Sim(w.lattices[c], [Particle(**{**p.__dict__, "cell": 0})])
        o.step(10)
        compare_state(g, o, "f32", cell=c, pid_offset=c)

"""GPU parity of the direct sweep with 2 or 4 consecutive cells per thread
(vector population accesses) against the FP64 oracle, and against the
one-cell sweep.

Lattices are chosen so that every code path of the grouped sweep runs: nx a
multiple of the group (vector loads and stores, odd-step x neighbours from
two aligned groups, periodic wrap at the row ends), nx a multiple of 2 but
not of 4 and odd nx (single lattices: cell by cell on odd steps; batches:
packed with element accesses inside the rows), a ragged last group, walls,
near-obstacle groups and split sweeps.
Tolerances as in test_gpu_parity: velocity relative L2 over fluid cells
1e-12 (FP64), 1e-5 (FP32), 1e-2 (FP16, BF16); flags and particle ids
bit-exact.
"""
import numpy as np
import pytest

import oracle
from lbm_inputs import Lattice, Particle, SplitMix64, quat_from_axis, shear_lattice

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


def rel_l2(a, b, mask):
    a, b = a[..., mask], b[..., mask]
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def compare(g, o, prec):
    _, ug, fg, pg, _ = g.fields(pdfs=False)
    _, uo, fo, po, _ = o.fields()
    assert np.array_equal(fg, fo), "flags differ"
    assert np.array_equal(pg, po), "particle ids differ"
    e = rel_l2(ug, uo, fo == 0)
    assert e <= TOL_U[prec], f"velocity rel L2 {e:.3e} > {TOL_U[prec]:.0e}"
    return e


def periodic_case(nx):
    lat = Lattice(nx, 18, 17, tau=0.7, periodic=(1, 1, 1), body_force=(2e-5, 0, 0))
    rng = SplitMix64(17)
    ps = [Particle(pos=(1.5, 9.2, 16.1), quat=quat_from_axis(rng.unit_vector()), semi_axes=(5.0, 2.5, 2.0),
                   vel=(0.02, -0.01, 0.03), omega=(0.0, 0.0, 0.01), density=20.0)]
    return lat, ps


@pytest.mark.parametrize("cpt", [2, 4])
@pytest.mark.parametrize("nx", [24, 22, 21])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_grouped_periodic_moving_body(lbm, prec, nx, cpt):
    """Fully periodic lattice (odd steps wrap on every face, x wrap inside a
    row of groups) with a body crossing the x seam."""
    if prec == "f64" and cpt == 4:
        pytest.skip("FP64 storage groups 1 or 2 cells")
    lat, ps = periodic_case(nx)
    g = lbm.Simulation(lat, ps, prec=prec)
    lbm.lbm_set_launch(g.h, 64, 0)
    lbm.lbm_set_cells_per_thread(g.h, cpt)
    assert lbm.lbm_get_info(g.h).cells_per_thread == cpt
    o = oracle.Sim(lat, ps)
    for c in (1, 4, 3):
        g.step(c)
        o.step(c)
        compare(g, o, prec)


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("cpt", [2, 4])
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_grouped_shear_three_bodies(lbm, prec, cpt, split):
    """Moving walls (wall-row groups) and three bodies (near-obstacle groups
    take the one-cell paths), fused and split sweeps, every parity."""
    lat = shear_lattice(40, 30, 26, 0.75, 0.015)
    rng = SplitMix64(23)
    ps = [Particle(pos=(12.0, 14.5, 12.5), quat=quat_from_axis(rng.unit_vector()), semi_axes=(7.0, 2.5, 2.5),
                   vel=(0.01, 0.0, -0.005), omega=(0.0, 0.004, 0.002), density=4.0),
          Particle(pos=(27.5, 13.0, 13.0), quat=quat_from_axis(rng.unit_vector()), semi_axes=(5.0, 2.0, 2.0),
                   vel=(-0.01, 0.002, 0.0), density=4.0),
          Particle(pos=(20.0, 21.5, 6.0), quat=quat_from_axis(rng.unit_vector()), semi_axes=(4.0, 2.0, 2.0),
                   omega=(0.01, 0.0, 0.0), density=4.0)]
    g = lbm.Simulation(lat, ps, prec=prec)
    lbm.lbm_set_launch(g.h, 128, 0)
    lbm.lbm_set_cells_per_thread(g.h, cpt)
    lbm.lbm_set_sweep_split(g.h, split)
    o = oracle.Sim(lat, ps)
    for c in (1, 4, 3, 12):
        g.step(c)
        o.step(c)
        compare(g, o, prec)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_grouped_equals_one_cell_sweep(lbm, prec):
    """With a fixed body the forces do not feed back into the fields, so the
    grouped sweeps must reproduce the one-cell sweep's populations to
    rounding: the arithmetic per cell is the same, but the compiler may fuse
    multiply-adds differently in the two code paths (the 16-bit forms take
    the same rounding bits per stored value)."""
    lat = shear_lattice(48, 22, 13, 0.8, 0.02)
    ps = [Particle(pos=(23.3, 10.6, 6.2), quat=quat_from_axis((0.6, 0.64, 0.48)), semi_axes=(8.0, 2.5, 2.5),
                   fixed=1)]
    tol = {"f64": 1e-13, "f32": 1e-6, "f16": 1e-3, "bf16": 1e-2}[prec]
    ref = None
    w = None
    for cpt in (1, 2, 4):
        if prec == "f64" and cpt == 4:
            continue
        g = lbm.Simulation(lat, ps, prec=prec)
        lbm.lbm_set_launch(g.h, 64, 0)
        lbm.lbm_set_cells_per_thread(g.h, cpt)
        g.step(7)
        _, _, fl, _, d = g.fields()
        g.close()
        if ref is None:
            ref, w = d, np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None]
            continue
        m = fl == 0
        e = np.linalg.norm((d - ref)[:, m]) / np.linalg.norm((ref - w)[:, m])
        assert e <= tol, f"cells per thread {cpt}: population offsets differ from the one-cell sweep by {e:.2e}"


def test_grouped_ragged_tail_and_batch(lbm):
    """A batch whose lattices have nx multiples of 4, of 2 only and odd, with
    lattice sizes that leave a ragged last group."""
    # every body spans less than half of each periodic extent (the minimum
    # image of a boundary link is then the link itself)
    lats = [shear_lattice(24, 13, 11, 0.8, 0.01), shear_lattice(22, 11, 9, 0.9, 0.02),
            shear_lattice(19, 12, 11, 0.7, 0.015)]
    rng = SplitMix64(31)
    ps = [Particle(pos=(11.3, 6.1, 4.2), quat=quat_from_axis(rng.unit_vector()), semi_axes=(4.0, 1.8, 1.8),
                   density=5.0, cell=0),
          Particle(pos=(10.2, 5.4, 3.3), quat=quat_from_axis(rng.unit_vector()), semi_axes=(3.0, 1.6, 1.6),
                   density=5.0, cell=1)]
    for cpt in (2, 4):
        g = lbm.Simulation(lats, ps, prec="f32")
        lbm.lbm_set_launch(g.h, 32, 0)
        lbm.lbm_set_cells_per_thread(g.h, cpt)
        g.step(9)
        for c, lat in enumerate(lats):
            own = [Particle(**{**p.__dict__, "cell": 0}) for p in ps if p.cell == c]
            o = oracle.Sim(lat, own)
            o.step(9)
            _, ug, fg, pg, _ = g.fields(cell=c, pdfs=False)
            _, uo, fo, po, _ = o.fields()
            assert np.array_equal(fg, fo)
            part = pg < 0xFFFFFFFC
            pg = pg.copy()
            pg[part] -= np.uint32(sum(1 for p in ps if p.cell < c))
            assert np.array_equal(pg, po)
            assert rel_l2(ug, uo, fo == 0) <= 1e-5
        g.close()


@pytest.mark.parametrize("split", [False, True])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_grouped_batch_unaligned_rows_equal_one_cell_sweep(lbm, prec, split):
    """In a batch, the odd steps of a lattice whose nx is not a multiple of
    the group run the packed path with element accesses for every group
    strictly inside a row, and cell by cell at the row ends: with fixed
    bodies (no feedback) the populations must match the one-cell sweep's to
    rounding, lattice by lattice."""
    lats = [shear_lattice(23, 14, 11, 0.8, 0.02), shear_lattice(30, 12, 9, 0.7, 0.015),
            shear_lattice(21, 13, 10, 0.9, 0.01)]
    ps = [Particle(pos=(11.3, 6.6, 5.2), quat=quat_from_axis((0.6, 0.64, 0.48)), semi_axes=(6.0, 2.5, 2.5),
                   fixed=1, cell=0),
          Particle(pos=(14.2, 5.4, 4.1), quat=quat_from_axis((0.0, 0.6, 0.8)), semi_axes=(5.0, 2.0, 2.0),
                   fixed=1, cell=1),
          Particle(pos=(9.7, 6.3, 4.8), quat=quat_from_axis((1.0, 0.0, 0.0)), semi_axes=(4.0, 2.2, 2.2),
                   fixed=1, cell=2)]
    tol = {"f64": 1e-13, "f32": 1e-6, "f16": 1e-3, "bf16": 1e-2}[prec]
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None]
    ref = None
    for cpt in (1, 2, 4):
        if prec == "f64" and cpt == 4:
            continue
        g = lbm.Simulation(lats, ps, prec=prec)
        lbm.lbm_set_launch(g.h, 64, 0)
        lbm.lbm_set_cells_per_thread(g.h, cpt)
        lbm.lbm_set_sweep_split(g.h, split)
        g.step(7)
        out = [g.fields(cell=c)[2::2] for c in range(len(lats))]
        g.close()
        if ref is None:
            ref = out
            continue
        for c, ((fl, d), (_, d0)) in enumerate(zip(out, ref)):
            m = fl == 0
            e = np.linalg.norm((d - d0)[:, m]) / np.linalg.norm((d0 - w)[:, m])
            assert e <= tol, f"cells per thread {cpt}, lattice {c}: offsets differ from the one-cell sweep by {e:.2e}"


def test_cells_per_thread_argument_errors(lbm):
    lat = shear_lattice(16, 10, 8, 0.8, 0.01)
    g = lbm.Simulation(lat, [], prec="f64")
    for bad in (0, 3, 4, 8, -1):
        with pytest.raises(lbm.LBMError):
            lbm.lbm_set_cells_per_thread(g.h, bad)
    lbm.lbm_set_cells_per_thread(g.h, 2)
    g.close()


@pytest.mark.parametrize("cpt", [1, 2, 4])
@pytest.mark.parametrize("grid", [0, 40])
def test_l2_prefetch_changes_nothing(lbm, cpt, grid):
    """The direct sweep's L2 prefetch is a hint: populations and flags
    bit-identical with and without it (in every sweep, or in the even- or the
    odd-step sweeps only), forces to the rounding of the FP64
    atomics' order (one tile per block, where a block prefetches the tile one
    wave ahead, and a persistent grid, where it prefetches its own next tile).
    The body is fixed, so the forces do not feed back into the fields."""
    lat = shear_lattice(64, 30, 26, 0.75, 0.015)
    rng = SplitMix64(41)
    ps = [Particle(pos=(30.0, 14.5, 12.5), quat=quat_from_axis(rng.unit_vector()), semi_axes=(7.0, 2.5, 2.5),
                   fixed=1)]
    out = []
    modes = (lbm.PREFETCH_OFF, lbm.PREFETCH_ALL, lbm.PREFETCH_EVEN, lbm.PREFETCH_ODD)
    for mode in modes:
        g = lbm.Simulation(lat, ps, prec="f32")
        lbm.lbm_set_cells_per_thread(g.h, cpt)
        lbm.lbm_set_launch(g.h, 128, grid)  # after the tile size is set
        lbm.lbm_set_sweep_prefetch(g.h, mode)
        info = lbm.lbm_get_info(g.h)
        assert info.sweep_prefetch_mode == mode
        assert (info.sweep_prefetch > 0) == (mode != lbm.PREFETCH_OFF)
        g.step(9)
        _, _, fl, _, d = g.fields()
        F, M = g.forces()
        out.append((fl, d, F, M))
        if mode == lbm.PREFETCH_ODD:
            for bad in (-1, 4):
                with pytest.raises(lbm.LBMError):
                    lbm.lbm_set_sweep_prefetch(g.h, bad)
            assert lbm.lbm_get_info(g.h).sweep_prefetch_mode == mode
        g.close()
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1], o[1])
        for a, b in zip(out[0][2:], o[2:]):
            assert np.allclose(a, b, rtol=1e-9, atol=1e-12)

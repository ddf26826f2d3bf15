"""Pins of the oracle's spherocylinder (the particle shape of Sec. 5.1, Fig.
Capsule: a cylinder of radius r with hemispherical end caps, total length L).

* mass and moments of inertia against an independent derivation: integration
  over slices normal to the axis, each a disc of radius rho(x) with area
  pi rho^2 and polar / diametral second moments pi rho^4 / 2 and pi rho^4 / 4
  (the oracle uses a cylinder + sphere decomposition and the parallel-axis
  theorem);
* the inside test with no cylindrical part equals the sphere (ellipsoid with
  three equal semi-axes) cell by cell;
* the obstacle mapping of a rotated spherocylinder equals a brute-force
  world-frame construction: distance from the cell centre to the axis segment
  from x_C - h t to x_C + h t (t the body axis), at most r;
* the mapped cell count converges to the analytic volume;
* a constant torque about a principal axis spins the body up at M / I.
"""
import math

import numpy as np
import pytest

import oracle
from lbm_inputs import Lattice, Particle, SplitMix64, quat_from_axis, SHAPE_SPHEROCYLINDER


def capsule(pos, quat, half_length, r, **kw):
    return Particle(pos=pos, quat=quat, semi_axes=(half_length, r, r), shape=SHAPE_SPHEROCYLINDER, **kw)


@pytest.mark.parametrize("half_length,r,density", [(8.0, 4.0, 1.195), (28.0, 4.0, 1.195), (4.0, 4.0, 2.0),
                                                   (10.0, 2.5, 1.0)])
def test_capsule_mass_inertia_by_slice_integration(half_length, r, density):
    integrate = pytest.importorskip("scipy.integrate")
    h = half_length - r

    def rho2(x):  # squared radius of the slice at axial position x
        t = max(abs(x) - h, 0.0)
        return max(r * r - t * t, 0.0)

    pts = [-h, h] if h > 0 else [0.0]
    kw = dict(points=pts, epsabs=0.0, epsrel=1e-13, limit=200)
    m = density * integrate.quad(lambda x: math.pi * rho2(x), -half_length, half_length, **kw)[0]
    i_axis = density * integrate.quad(lambda x: math.pi * rho2(x) ** 2 / 2, -half_length, half_length, **kw)[0]
    i_trans = density * integrate.quad(lambda x: math.pi * rho2(x) ** 2 / 4 + x * x * math.pi * rho2(x),
                                       -half_length, half_length, **kw)[0]
    rec = oracle.particle_records([capsule((0, 0, 0), (1, 0, 0, 0), half_length, r, density=density)])[0]
    mo, I = oracle.mass_inertia(rec)
    assert mo == pytest.approx(m, rel=1e-11)
    assert I[0] == pytest.approx(i_axis, rel=1e-11)
    assert I[1] == pytest.approx(i_trans, rel=1e-11)
    assert I[2] == I[1]


@pytest.mark.parametrize("seed", [1, 2])
def test_capsule_without_cylinder_is_the_sphere(seed):
    rng = SplitMix64(seed)
    dims, per = (16, 16, 16), np.array([1, 1, 1], np.int32)
    for _ in range(3):
        pos = (7.5 + rng.uniform() - 0.5, 8.0 + rng.uniform() - 0.5, 7.7 + rng.uniform() - 0.5)
        q = quat_from_axis(rng.unit_vector())
        cap = oracle.particle_records([capsule(pos, q, 4.6, 4.6)])[0]
        sph = oracle.particle_records([Particle(pos=pos, quat=q, semi_axes=(4.6, 4.6, 4.6))])[0]
        for k in range(16):
            for j in range(16):
                for i in range(16):
                    assert oracle.inside(cap, dims, per, i, j, k) == oracle.inside(sph, dims, per, i, j, k)


def _segment_distance2(cells, c, t, h):
    """Squared distance from each cell centre to the segment c + s t, |s| <= h."""
    d = cells - c
    s = np.clip(d @ t, -h, h)
    e = d - s[:, None] * t[None, :]
    return np.einsum("ij,ij->i", e, e)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_capsule_mapping_matches_world_frame_construction(seed):
    rng = SplitMix64(seed)
    n = 30
    lat = Lattice(n, n, n, periodic=(0, 0, 0))
    half_length, r = 9.0, 3.2
    pos = (14.3 + rng.uniform(), 14.8 + rng.uniform(), 15.1 + rng.uniform())
    q = quat_from_axis(rng.unit_vector())
    s = oracle.Sim(lat, [capsule(pos, q, half_length, r)])
    _, _, fl, pid, _ = s.fields()
    R = oracle.quat_to_matrix(np.array(q) / np.linalg.norm(q))
    t = R[:, 0]  # body x axis in world coordinates
    idx = np.arange(n ** 3)
    cells = np.stack([idx % n, (idx // n) % n, idx // (n * n)], axis=1).astype(float)
    d2 = _segment_distance2(cells, np.array(pos), t, half_length - r)
    inner = np.all((cells >= 1) & (cells <= n - 2), axis=1)
    clear = np.abs(d2 - r * r) > 1e-9
    exp = np.where(d2 <= r * r, 0, 0xFFFFFFFF).astype(np.uint32)
    ok = inner & clear
    assert np.array_equal(pid[ok], exp[ok])
    assert np.array_equal(fl[ok], np.where(exp[ok] == 0, 2, 0).astype(fl.dtype))
    assert (pid == 0).sum() > 200


def test_capsule_mapped_volume_converges():
    rng = SplitMix64(6)
    errs = []
    for scale in (1.0, 2.0):
        half_length, r = 7.0 * scale, 2.5 * scale
        n = int(2 * half_length + 6)
        lat = Lattice(n, n, n, periodic=(1, 1, 1))
        p = capsule((n / 2 - 0.37, n / 2 + 0.21, n / 2 + 0.05), quat_from_axis(rng.unit_vector()), half_length, r)
        s = oracle.Sim(lat, [p])
        _, _, fl, _, _ = s.fields()
        vol = math.pi * r * r * (2 * half_length - 2 * r) + 4 / 3 * math.pi * r ** 3
        errs.append(abs((fl == 2).sum() / vol - 1))
    assert errs[1] < 0.02


def test_capsule_spins_up_at_torque_over_inertia():
    rec = oracle.particle_records([capsule((0, 0, 0), (1, 0, 0, 0), 8.0, 4.0, density=1.195)])[0]
    m, I = oracle.mass_inertia(rec)
    L = np.zeros(3)
    M = np.array([0.0, 0.0, 3.0])  # about body z, a transverse principal axis
    for _ in range(5):
        oracle.rigid_body_step(rec, L, np.zeros(3), M)
    assert rec[12] == pytest.approx(5 * 3.0 / I[2], rel=1e-13)
    assert abs(rec[10]) < 1e-15 and abs(rec[11]) < 1e-15

"""Parity at the full sizes of the benchmarked workloads, in the launch
configuration the bench times (the autotuner's choice):

* 256x128x128 shear flow with the a = 24, b = 3 spheroid, started from the
  Couette profile: 20 steps of the CUDA path in FP32, FP16 and BF16 storage
  against 20 steps of the FP64 oracle on the whole lattice (OpenMP over the
  host cores): flags and particle ids bit-exact, velocity relative L2 1e-5 /
  1e-2 / 2e-2, force and torque on the hydrodynamic scales mu gamma a b and
  mu gamma a^2 b;
* the batch of 512 shear cells: one batched context stepped 10 times, six
  seeded lattices of it stepped alone by the oracle and compared cell by cell;
* the 512x256x256 suspension of 2,000 spheroids (too large for the
  brute-force oracle mapping, O(cells x bodies)): after 20 steps, the particle
  ids in the boxes of 12 seeded bodies equal the oracle's inside test applied
  to the poses the CUDA path reports (the mapping is exact given the pose).
"""
import os

import numpy as np
import pytest

import oracle
from lbm_inputs import (Particle, SplitMix64, batched_shear, fibre_suspension, large_shear, PID_FLUID,
                        PID_WALL)

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
CX = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0], dtype=float)
STEPS = 20


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
    y = np.arange(lat.ny, dtype=float)
    ux = lat.wall_u_lo[0] + (lat.wall_u_hi[0] - lat.wall_u_lo[0]) * (y - 0.5) / (lat.ny - 2.0)
    cu = np.outer(CX, ux)
    feq = W[:, None] * lat.rho0 * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * ux[None, :] ** 2)
    n = lat.nx * lat.ny * lat.nz
    return np.ascontiguousarray(feq[:, (np.arange(n) // lat.nx) % lat.ny])


def rel_l2(a, b, mask):
    a, b = a[..., mask], b[..., mask]
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def large_reference():
    w = large_shear(seed=1)
    lat = w.lattices[0]
    o = oracle.Sim(lat, w.particles, openmp=True, threads=os.cpu_count() or 1)
    o.set_pdfs(couette_pdfs(lat))
    o.step(STEPS)
    _, u, fl, pid, _ = o.fields()
    F, M = o.forces()
    return w, u, fl, pid, F, M


@pytest.mark.parametrize("prec,tol_u,tol_f", [("f32", 1e-5, 1e-4), ("f16", 1e-2, 2e-2), ("bf16", 1e-2, 5e-2)])
def test_large_shear_full_size(lbm, large_reference, prec, tol_u, tol_f):
    w, uo, fo, po, Fo, Mo = large_reference
    lat = w.lattices[0]
    g = lbm.Simulation(lat, w.particles, prec=prec)
    g.set_pdfs(couette_pdfs(lat))
    lbm.lbm_autotune(g.h)
    g.step(STEPS)
    _, ug, fg, pg, _ = g.fields(0, pdfs=False)
    Fg, Mg = g.forces()
    info = g.info()
    g.close()
    assert np.array_equal(fg, fo) and np.array_equal(pg, po)
    e = rel_l2(ug, uo, fo == 0)
    a, b = w.particles[0].semi_axes[0], w.particles[0].semi_axes[1]
    mu = lat.rho0 * (lat.tau - 0.5) / 3.0
    gamma = abs(lat.wall_u_hi[0] - lat.wall_u_lo[0]) / (lat.ny - 2.0)
    eF = np.abs(Fg - Fo).max() / (mu * gamma * a * b)
    eM = np.abs(Mg - Mo).max() / (mu * gamma * a * a * b)
    print(f"{prec} full size: launch block {info.sweep_block} grid {info.sweep_grid} split {info.sweep_split}; "
          f"velocity rel L2 {e:.2e}, |dF|/(mu g a b) {eF:.2e}, |dM|/(mu g a^2 b) {eM:.2e}")
    assert e <= tol_u and eF <= tol_f and eM <= tol_f


def test_batched_full_size_sampled_lattices(lbm):
    steps = 10
    w = batched_shear(seed=1)
    g = lbm.Simulation(w.lattices, w.particles, prec="f32")
    lbm.lbm_autotune(g.h)
    g.step(steps)
    rng = SplitMix64(77)
    picks = sorted({int(rng.uniform() * len(w.lattices)) for _ in range(6)})
    owner = {p.cell: i for i, p in enumerate(w.particles)}
    for c in picks:
        lat = w.lattices[c]
        mine = [Particle(**{**p.__dict__, "cell": 0}) for p in w.particles if p.cell == c]
        o = oracle.Sim(lat, mine)
        o.step(steps)
        _, ug, fg, pg, _ = g.fields(c, pdfs=False)
        _, uo, fo, po, _ = o.fields()
        part = pg < PID_WALL
        pg = pg.copy()
        pg[part] -= np.uint32(owner.get(c, 0))
        assert np.array_equal(fg, fo), c
        assert np.array_equal(pg, po), c
        assert rel_l2(ug, uo, fo == 0) <= 1e-5, c
    g.close()


def test_fibre_full_size_mapping_of_sampled_bodies(lbm):
    w = fibre_suspension(seed=1)
    lat = w.lattices[0]
    dims, per = (lat.nx, lat.ny, lat.nz), np.array(lat.periodic, np.int32)
    g = lbm.Simulation(lat, w.particles, prec="f32")
    lbm.lbm_autotune(g.h)
    g.step(STEPS)
    recs = g.particles()
    pid = lbm.lbm_get_fields(g.h, lat.ncells, 0, rho=False, u=False, flags=False, pid=True)["pid"]
    g.close()
    rng = SplitMix64(78)
    picks = sorted({int(rng.uniform() * len(recs)) for _ in range(12)})
    centres = recs[:, 0:3]
    reach = recs[:, 13] + 3.0
    for p in picks:
        lo = np.floor(centres[p] - reach[p]).astype(int)
        hi = np.ceil(centres[p] + reach[p]).astype(int)
        kk, jj, ii = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(max(lo[1], 0), min(hi[1], dims[1] - 1) + 1),
                                 np.arange(lo[0], hi[0] + 1), indexing="ij")
        ii, jj, kk = ii.ravel() % dims[0], jj.ravel(), kk.ravel() % dims[2]
        x = ii + dims[0] * (jj + dims[1] * kk)
        fluid_region = ~((pid[x] >= PID_WALL) & (pid[x] < PID_FLUID))
        cells = np.stack([ii, jj, kk], axis=1).astype(float)
        exp = np.full(len(x), PID_FLUID, np.uint32)
        d = centres - centres[p]
        for a in (0, 2):  # periodic x and z: minimum image
            d[:, a] -= dims[a] * np.round(d[:, a] / dims[a])
        # every body that can reach into the box (its corners lie sqrt(3) reach from the centre); ascending
        # order: the lowest index wins
        for q in np.nonzero(np.linalg.norm(d, axis=1) <= np.sqrt(3.0) * reach[p] + reach)[0]:
            # cells that may lie inside body q: within b + 2 of its axis segment
            dq = cells - centres[q]
            for a in (0, 2):
                dq[:, a] -= dims[a] * np.round(dq[:, a] / dims[a])
            R = oracle.quat_to_matrix(recs[q, 3:7] / np.linalg.norm(recs[q, 3:7]))
            s_ax = np.clip(dq @ R[:, 0], -recs[q, 13], recs[q, 13])
            near = np.linalg.norm(dq - s_ax[:, None] * R[:, 0][None, :], axis=1) <= recs[q, 14:16].max() + 2.0
            for c in np.nonzero(near & (exp == PID_FLUID) & fluid_region)[0]:
                if oracle.inside(recs[q], dims, per, int(ii[c]), int(jj[c]), int(kk[c])):
                    exp[c] = q
        ok = fluid_region
        bad = np.nonzero(pid[x][ok] != exp[ok])[0]
        assert len(bad) == 0, (p, cells[ok][bad[:5]], pid[x][ok][bad[:5]], exp[ok][bad[:5]])
        assert (exp == p).sum() > 50

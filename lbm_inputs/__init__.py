"""Seeded synthetic inputs for the LBM / moving-particle workloads.

This module is shared by the CPU oracle tests, the GPU parity tests, the bench
and the smoke entry.  It holds none of the lattice Boltzmann arithmetic: it only
draws random numbers and turns them into lattice descriptions and particle poses
(position, unit quaternion, semi-axes), which both implementations receive as
identical doubles.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) and unit vectors from
Marsaglia's method (Ann. Math. Stat. 43, 1972).

Workload shapes follow the five shear-cell workloads of the paper's fully
resolved particle model (Sec. 4): a D3Q19 TRT lattice with moving walls at
y = 0 and y = ny-1, periodic in x and z, holding prolate spheroids.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

MASK64 = (1 << 64) - 1

# Particle-id codes of non-fluid, non-particle cells (match the C interface).
PID_FLUID = 0xFFFFFFFF
PID_WALL_YLO = 0xFFFFFFFE
PID_WALL_YHI = 0xFFFFFFFD
PID_WALL = 0xFFFFFFFC
SHAPE_ELLIPSOID, SHAPE_SPHEROCYLINDER = 0, 1


class SplitMix64:
    """SplitMix64 generator; ``uniform()`` maps the top 53 bits to [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def unit_vector(self) -> Tuple[float, float, float]:
        """Uniform point on the unit sphere (Marsaglia 1972 rejection method)."""
        while True:
            v1 = 2.0 * self.uniform() - 1.0
            v2 = 2.0 * self.uniform() - 1.0
            s = v1 * v1 + v2 * v2
            if s < 1.0:
                r = 2.0 * math.sqrt(1.0 - s)
                return (v1 * r, v2 * r, 1.0 - 2.0 * s)


def quat_from_axis(t: Sequence[float]) -> Tuple[float, float, float, float]:
    """Unit quaternion (w, x, y, z) of the shortest rotation taking the body x
    axis onto the unit vector ``t``: q ~ (1 + t_x, e_x cross t)."""
    tx, ty, tz = t
    w, x, y, z = 1.0 + tx, 0.0, -tz, ty
    n = math.sqrt(w * w + x * x + y * y + z * z)
    if n < 1e-12:            # t = -e_x: half turn about z
        return (0.0, 0.0, 0.0, 1.0)
    return (w / n, x / n, y / n, z / n)


def axis_from_quat(q: Sequence[float]) -> Tuple[float, float, float]:
    """Image of the body x axis under the rotation q (first column of R)."""
    w, x, y, z = q
    return (1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y + w * z), 2.0 * (x * z - w * y))


@dataclass
class Lattice:
    """One lattice: size, relaxation, periodic axes, wall speeds (lattice
    units); free_slip[a] turns the wall layers of non-periodic axis a into
    free-slip walls."""
    nx: int
    ny: int
    nz: int
    tau: float = 0.8
    magic: float = 3.0 / 16.0
    rho0: float = 1.0
    periodic: Tuple[int, int, int] = (1, 0, 1)
    wall_u_lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    wall_u_hi: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    body_force: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    free_slip: Tuple[int, int, int] = (0, 0, 0)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class Particle:
    """Rigid body: centre, orientation, velocities, semi-axes (body x,y,z).
    shape 0: ellipsoid with those semi-axes; shape 1: spherocylinder of total
    length L and radius r along body x, semi_axes = (L/2, r, r)."""
    pos: Tuple[float, float, float]
    quat: Tuple[float, float, float, float]
    semi_axes: Tuple[float, float, float]
    vel: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    omega: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    density: float = 2.0
    ext_force: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    ext_torque: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    cell: int = 0
    fixed: int = 0
    shape: int = 0


@dataclass
class Workload:
    name: str
    lattices: List[Lattice]
    particles: List[Particle]
    steps: int
    extra: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return sum(l.ncells for l in self.lattices)


def shear_lattice(nx: int, ny: int, nz: int, tau: float, uw: float) -> Lattice:
    """Couette cell: wall y=0 moves at -uw in x, wall y=ny-1 at +uw."""
    return Lattice(nx, ny, nz, tau=tau, periodic=(1, 0, 1),
                   wall_u_lo=(-uw, 0.0, 0.0), wall_u_hi=(uw, 0.0, 0.0))


def centre(lat: Lattice) -> Tuple[float, float, float]:
    return ((lat.nx - 1) / 2.0, (lat.ny - 1) / 2.0, (lat.nz - 1) / 2.0)


# Particle-to-fluid density ratio of every workload.  The explicit
# momentum-exchange coupling goes unstable for light bodies (the spin about the
# symmetry axis of a thin spheroid diverges at density ratio 1 with b = 2);
# ratio 2 is stable for minor semi-axes b >= 1.5 at tau = 0.8.
DENSITY = 2.0
# The batched cells draw tau down to 0.6 with b down to 1.5, where ratios 2
# and 3 still diverge (FP64 oracle runs of the least viscous, thinnest cells
# blow up after 250 and 850 steps); ratio 5 stays bounded over 3,000 steps.
BATCH_DENSITY = 5.0


def spheroid_at_centre(lat: Lattice, a: float, b: float, rng: SplitMix64,
                       density: float = DENSITY) -> Particle:
    return Particle(pos=centre(lat), quat=quat_from_axis(rng.unit_vector()),
                    semi_axes=(a, b, b), density=density)


def small_shear(seed: int = 1, n: int = 32, steps: int = 200) -> Workload:
    """FP64 oracle-size case: 32^3, tau 0.8, walls +-0.01, spheroid (8,2,2)."""
    rng = SplitMix64(seed)
    lat = shear_lattice(n, n, n, 0.8, 0.01)
    p = spheroid_at_centre(lat, 8.0, 2.0, rng)
    return Workload(f"shear{n}^3_spheroid8x2x2_fp64", [lat], [p], steps)


def large_shear(seed: int = 1, steps: int = 20000) -> Workload:
    """Scale case: 256x128x128, tau 0.8, walls +-0.02, spheroid a=24, b=3."""
    rng = SplitMix64(seed)
    lat = shear_lattice(256, 128, 128, 0.8, 0.02)
    p = spheroid_at_centre(lat, 24.0, 3.0, rng)
    return Workload("shear256x128x128_spheroid24x3x3", [lat], [p], steps)


def batched_shear(seed: int = 1, ncell: int = 512, steps: int = 5000) -> Workload:
    """Batched case: independent shear cells with drawn sizes and parameters.

    nx ~ U{48..96}, ny, nz ~ U{48..64}; aspect ~ U[2,10], minor semi-axis
    b ~ U[1.5,4] (redrawn until 2a+4 <= min(nx, ny-2, nz)); wall speed
    ~ U[0.005,0.03]; tau ~ U[0.6,1.2]; seeded orientation at the cell centre;
    body density ratio BATCH_DENSITY.
    """
    rng = SplitMix64(seed)
    lats, parts = [], []
    for c in range(ncell):
        nx = rng.randint(48, 96)
        ny = rng.randint(48, 64)
        nz = rng.randint(48, 64)
        uw = rng.uniform_range(0.005, 0.03)
        tau = rng.uniform_range(0.6, 1.2)
        lat = shear_lattice(nx, ny, nz, tau, uw)
        while True:
            aspect = rng.uniform_range(2.0, 10.0)
            b = rng.uniform_range(1.5, 4.0)
            a = aspect * b
            if 2.0 * a + 4.0 <= min(nx, ny - 2, nz):
                break
        p = spheroid_at_centre(lat, a, b, rng, density=BATCH_DENSITY)
        p.cell = c
        lats.append(lat)
        parts.append(p)
    return Workload(f"batched{ncell}_shear_cells", lats, parts, steps)


def _segment_distance(p0, d0, p1, d1) -> float:
    """Distance between segments p0 + s d0 and p1 + t d1, s, t in [-1, 1]."""
    def dot(u, v):
        return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]
    r = [p0[i] - p1[i] for i in range(3)]
    a, e, f = dot(d0, d0), dot(d1, d1), dot(d1, r)
    b, c = dot(d0, d1), dot(d0, r)
    denom = a * e - b * b
    s = 0.0 if denom < 1e-12 else max(-1.0, min(1.0, (b * f - c * e) / denom))
    t = max(-1.0, min(1.0, (b * s + f) / e))
    s = max(-1.0, min(1.0, (b * t - c) / a))
    d = [r[i] + s * d0[i] - t * d1[i] for i in range(3)]
    return math.sqrt(dot(d, d))


def fibre_suspension(seed: int = 1, nx: int = 512, ny: int = 256, nz: int = 256,
                     count: int = 2000, a: float = 15.0, b: float = 1.5,
                     uw: float = 0.02, tau: float = 0.8, gap: float = 2.0,
                     steps: int = 2000) -> Workload:
    """Fibre suspension: ``count`` prolate spheroids (a, b, b) at seeded uniform
    positions and orientations, no two closer than ``gap`` cells.

    A prolate spheroid lies inside the capsule whose axis segment is
    [-(a-b), a-b] with radius b, so two spheroids are disjoint if their
    segments are more than 2b apart; placement is rejected otherwise.
    Positions keep the whole body at least 2 cells off the walls.
    """
    rng = SplitMix64(seed)
    lat = shear_lattice(nx, ny, nz, tau, uw)
    parts: List[Particle] = []
    segs = []
    half = a - b
    tries = 0
    while len(parts) < count:
        tries += 1
        if tries > 200 * count:
            raise RuntimeError("fibre placement did not converge")
        t = rng.unit_vector()
        pos = (rng.uniform_range(0.0, nx), rng.uniform_range(0.0, ny), rng.uniform_range(0.0, nz))
        ext_y = math.sqrt((a * t[1]) ** 2 + b * b * (1.0 - t[1] * t[1]))
        if pos[1] - ext_y < 3.0 or pos[1] + ext_y > ny - 4.0:
            continue
        d = (t[0] * half, t[1] * half, t[2] * half)
        ok = True
        for (q, e) in segs:
            # minimum image in the periodic x and z directions
            rx = pos[0] - q[0]
            rz = pos[2] - q[2]
            sx = -nx * round(rx / nx)
            sz = -nz * round(rz / nz)
            if abs(rx + sx) > 2 * a + gap or abs(pos[1] - q[1]) > 2 * a + gap or abs(rz + sz) > 2 * a + gap:
                continue
            qq = (q[0] - sx, q[1], q[2] - sz)
            if _segment_distance(pos, d, qq, e) <= 2.0 * b + gap:
                ok = False
                break
        if not ok:
            continue
        segs.append((pos, d))
        parts.append(Particle(pos=pos, quat=quat_from_axis(t), semi_axes=(a, b, b),
                              density=DENSITY))
    return Workload(f"suspension{nx}x{ny}x{nz}_{count}_spheroids", [lat], parts, steps)


def random_populations_seed(seed: int, n: int) -> List[float]:
    """Uniform [0,1) stream of length n (for perturbing populations in tests)."""
    rng = SplitMix64(seed)
    return [rng.uniform() for _ in range(n)]

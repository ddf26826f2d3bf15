"""CPU FP64 oracle of the lattice Boltzmann / moving-particle model.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the GPU library (``paper_1503_06869_gb300``) and never imports it.

``build()`` compiles ``lbm_oracle.c`` with gcc into ``_build/liblbm_oracle.so``
(``-ffp-contract=off`` so that each product and sum rounds separately, as the
bit-exact obstacle mapping requires), plus an OpenMP variant used only for
timing the CPU baseline.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "lbm_oracle.c")
HDR = os.path.join(HERE, "lbm_oracle.h")
PSTRIDE = 26
SHAPE_ELLIPSOID, SHAPE_SPHEROCYLINDER = 0, 1
Q = 19

_lock = threading.Lock()
_libs = {}


def _lib_path(openmp: bool) -> str:
    return os.path.join(BUILD, "liblbm_oracle_omp.so" if openmp else "liblbm_oracle.so")


def build(openmp: bool = False, force: bool = False) -> str:
    """Compile the oracle (if stale) and return the shared-library path."""
    out = _lib_path(openmp)
    os.makedirs(BUILD, exist_ok=True)
    src_m = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < src_m:
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
               "-shared", "-o", tmp, SRC, "-lm"]
        if openmp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _declare(lib):
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                               ip, dp, dp, dp]
    lib.orc_destroy.argtypes = [C.c_void_p]
    lib.orc_set_particles.argtypes = [C.c_void_p, dp, C.c_int]
    lib.orc_step.argtypes = [C.c_void_p, C.c_int]
    lib.orc_step_count.restype = C.c_long
    lib.orc_step_count.argtypes = [C.c_void_p]
    lib.orc_get_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]
    lib.orc_set_pdfs.argtypes = [C.c_void_p, C.c_void_p]
    lib.orc_get_forces.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_get_wall_forces.argtypes = [C.c_void_p, C.c_void_p]
    lib.orc_get_particles.argtypes = [C.c_void_p, C.c_void_p]
    lib.orc_get_links.restype = C.c_int
    lib.orc_get_links.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_lattice.argtypes = [C.c_void_p] * 5
    lib.orc_omega_odd.restype = C.c_double
    lib.orc_omega_odd.argtypes = [C.c_double, C.c_double]
    lib.orc_equilibrium.argtypes = [C.c_double, C.c_void_p, C.c_double, C.c_void_p]
    lib.orc_collide_cell.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    lib.orc_set_momentum_stabilisation.argtypes = [C.c_void_p, C.c_int]
    lib.orc_set_free_slip.argtypes = [C.c_void_p, C.c_void_p]
    lib.orc_inside.restype = C.c_int
    lib.orc_inside.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                               C.c_int, C.c_int]
    lib.orc_quat_to_matrix.argtypes = [C.c_void_p, C.c_void_p]
    lib.orc_rigid_body_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.orc_particle_mass_inertia.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    return lib


def lib(openmp: bool = False):
    with _lock:
        if openmp not in _libs:
            _libs[openmp] = _declare(C.CDLL(build(openmp)))
        return _libs[openmp]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def particle_records(particles) -> np.ndarray:
    """Pack particle objects (pos, quat, vel, omega, semi_axes, density,
    ext_force, ext_torque, fixed, cell, shape) into the oracle's record array."""
    out = np.zeros((len(particles), PSTRIDE), dtype=np.float64)
    for i, p in enumerate(particles):
        out[i, 0:3] = p.pos
        out[i, 3:7] = p.quat
        out[i, 7:10] = p.vel
        out[i, 10:13] = p.omega
        out[i, 13:16] = p.semi_axes
        out[i, 16] = p.density
        out[i, 17:20] = p.ext_force
        out[i, 20:23] = p.ext_torque
        out[i, 23] = float(p.fixed)
        out[i, 24] = float(p.cell)
        out[i, 25] = float(getattr(p, "shape", SHAPE_ELLIPSOID))
    return out


def lattice_tables():
    L = lib()
    cx = np.zeros(Q, np.int32)
    cy = np.zeros(Q, np.int32)
    cz = np.zeros(Q, np.int32)
    w = np.zeros(Q, np.float64)
    opp = np.zeros(Q, np.int32)
    L.orc_lattice(_ptr(cx), _ptr(cy), _ptr(cz), _ptr(w), _ptr(opp))
    return np.stack([cx, cy, cz], axis=1), w, opp


def omega_odd(tau: float, magic: float) -> float:
    return lib().orc_omega_odd(tau, magic)


def equilibrium(rho: float, u, rho0: float = 1.0) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    lib().orc_equilibrium(rho, _ptr(u), rho0, _ptr(out))
    return out


def collide_cell(f, omega: float, omega_o: float, rho0: float = 1.0, g=(0.0, 0.0, 0.0), ubar=(0.0, 0.0, 0.0)):
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    ub = np.ascontiguousarray(ubar, dtype=np.float64)
    out = np.zeros(Q)
    lib().orc_collide_cell(_ptr(f), omega, omega_o, rho0, _ptr(g), _ptr(ub), _ptr(out))
    return out


def quat_to_matrix(q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.zeros(9)
    lib().orc_quat_to_matrix(_ptr(q), _ptr(R))
    return R.reshape(3, 3)


def inside(record, dims, periodic, i, j, k) -> bool:
    record = np.ascontiguousarray(record, dtype=np.float64)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    return bool(lib().orc_inside(_ptr(record), dims[0], dims[1], dims[2], _ptr(per), i, j, k))


def rigid_body_step(record, L, F, M):
    """Advance one record in place (and its angular momentum L) by one step."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    lib().orc_rigid_body_step(_ptr(record), _ptr(L), _ptr(F), _ptr(M))


def mass_inertia(record):
    record = np.ascontiguousarray(record, dtype=np.float64)
    m = np.zeros(1)
    I = np.zeros(3)
    lib().orc_particle_mass_inertia(_ptr(record), _ptr(m), _ptr(I))
    return float(m[0]), I


class Sim:
    """One lattice simulated by the oracle (see ``lbm_oracle.h``)."""

    def __init__(self, lat, particles=(), openmp: bool = False, threads: int = 1):
        self._L = lib(openmp)
        if openmp:
            self._L.orc_set_threads(threads)
        self.lat = lat
        self.dims = (lat.nx, lat.ny, lat.nz)
        self.n = lat.nx * lat.ny * lat.nz
        per = np.array(lat.periodic, np.int32)
        wl = np.array(lat.wall_u_lo, np.float64)
        wh = np.array(lat.wall_u_hi, np.float64)
        g = np.array(lat.body_force, np.float64)
        self._keep = (per, wl, wh, g)
        self.h = self._L.orc_create(lat.nx, lat.ny, lat.nz, lat.tau, lat.magic, lat.rho0,
                                    per.ctypes.data_as(C.POINTER(C.c_int)),
                                    wl.ctypes.data_as(C.POINTER(C.c_double)),
                                    wh.ctypes.data_as(C.POINTER(C.c_double)),
                                    g.ctypes.data_as(C.POINTER(C.c_double)))
        self.np = 0
        fs = np.array(getattr(lat, "free_slip", (0, 0, 0)), np.int32)
        if fs.any():
            self._L.orc_set_free_slip(self.h, _ptr(fs))
        if len(particles):
            self.set_particles(particles)

    def set_momentum_stabilisation(self, enable: bool = True):
        self._L.orc_set_momentum_stabilisation(self.h, 1 if enable else 0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.orc_destroy(h)
            self.h = None

    def set_particles(self, particles):
        rec = particles if isinstance(particles, np.ndarray) else particle_records(particles)
        rec = np.ascontiguousarray(rec, dtype=np.float64)
        self.np = rec.shape[0]
        self._L.orc_set_particles(self.h, rec.ctypes.data_as(C.POINTER(C.c_double)), self.np)

    def step(self, n: int = 1):
        self._L.orc_step(self.h, n)

    @property
    def t(self) -> int:
        return self._L.orc_step_count(self.h)

    def fields(self):
        """(rho[n], u[3,n], flags[n], pid[n], pdfs[19,n]) in cell order idx = x + nx(y + ny z)."""
        n = self.n
        rho = np.zeros(n)
        u = np.zeros((3, n))
        fl = np.zeros(n, np.uint8)
        pid = np.zeros(n, np.uint32)
        pdf = np.zeros((Q, n))
        self._L.orc_get_fields(self.h, _ptr(rho), _ptr(u), _ptr(fl), _ptr(pid), _ptr(pdf))
        return rho, u, fl, pid, pdf

    def set_pdfs(self, pdfs):
        pdfs = np.ascontiguousarray(pdfs, dtype=np.float64).reshape(Q, self.n)
        self._L.orc_set_pdfs(self.h, _ptr(pdfs))

    def forces(self):
        F = np.zeros((self.np, 3))
        M = np.zeros((self.np, 3))
        if self.np:
            self._L.orc_get_forces(self.h, _ptr(F), _ptr(M))
        return F, M

    def wall_forces(self):
        f = np.zeros(6)
        self._L.orc_get_wall_forces(self.h, _ptr(f))
        return f.reshape(2, 3)

    def particles(self) -> np.ndarray:
        out = np.zeros((self.np, PSTRIDE))
        if self.np:
            self._L.orc_get_particles(self.h, _ptr(out))
        return out

    def links(self):
        cnt = self._L.orc_get_links(self.h, None, None, None, 0)
        cell = np.zeros(cnt, np.int32)
        q = np.zeros(cnt, np.int8)
        pid = np.zeros(cnt, np.uint32)
        self._L.orc_get_links(self.h, _ptr(cell), _ptr(q), _ptr(pid), cnt)
        return cell, q, pid

"""ctypes binding of the C interface in ``include/lbm.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_lib/liblbm_gb300.so``.  Loading fails loudly when the library is missing;
there is no CPU fallback.  PyTorch supplies device memory (caching allocator)
and the stream.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblbm_gb300.so")

Q = 19
LBM_OK, LBM_ERR_ARG, LBM_ERR_STATE, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NUMERIC, LBM_ERR_TIMEOUT, \
    LBM_ERR_UNSUPPORTED = range(8)
LBM_F64, LBM_F32, LBM_F16_OFFSET, LBM_BF16_OFFSET = range(4)
PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16_OFFSET, "bf16": LBM_BF16_OFFSET}
LBM_PID_FLUID = 0xFFFFFFFF
LBM_PID_WALL_YLO = 0xFFFFFFFE
LBM_PID_WALL_YHI = 0xFFFFFFFD
LBM_PID_WALL = 0xFFFFFFFC

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

D3 = C.c_double * 3


class lbm_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("magic", C.c_double), ("rho0", C.c_double),
                ("periodic", C.c_int * 3),
                ("wall_u_lo", D3), ("wall_u_hi", D3), ("body_force", D3),
                ("prec", C.c_int),
                ("cuda_stream", C.c_void_p),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("user", C.c_void_p),
                ("free_slip", C.c_int * 3)]


class lbm_particle(C.Structure):
    _fields_ = [("pos", D3), ("quat", C.c_double * 4), ("vel", D3), ("omega", D3),
                ("semi_axes", D3), ("density", C.c_double), ("ext_force", D3),
                ("ext_torque", D3), ("cell", C.c_int), ("fixed", C.c_int), ("shape", C.c_int)]


class lbm_info(C.Structure):
    _fields_ = [("ncells_total", C.c_longlong), ("nfluid_hint", C.c_longlong),
                ("nlattices", C.c_int), ("nparticles", C.c_int), ("steps_done", C.c_longlong),
                ("device_bytes", C.c_size_t), ("sweep_grid", C.c_int), ("sweep_block", C.c_int),
                ("bytes_per_population", C.c_int), ("sweep_split", C.c_int),
                ("remap_fused", C.c_int), ("remap_grid", C.c_int),
                ("cells_per_thread", C.c_int), ("device", C.c_int), ("sweep_prefetch", C.c_int),
                ("sweep_prefetch_mode", C.c_int)]


# name -> (restype, argtypes) for every entry point of include/lbm.h
SIGNATURES = {
    "lbm_create": (C.c_int, [C.POINTER(lbm_grid_desc), C.POINTER(C.c_void_p)]),
    "lbm_create_batch": (C.c_int, [C.POINTER(lbm_grid_desc), C.c_int, C.POINTER(C.c_void_p)]),
    "lbm_set_particles": (C.c_int, [C.c_void_p, C.POINTER(lbm_particle), C.c_int]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_sync": (C.c_int, [C.c_void_p]),
    "lbm_get_forces": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "lbm_get_wall_forces": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lbm_get_particles": (C.c_int, [C.c_void_p, C.POINTER(lbm_particle), C.c_int]),
    "lbm_set_external": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "lbm_get_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "lbm_set_pdfs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lbm_get_links": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                C.POINTER(C.c_int)]),
    "lbm_get_links_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                        C.c_void_p]),
    "lbm_get_info": (C.c_int, [C.c_void_p, C.POINTER(lbm_info)]),
    "lbm_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "lbm_set_cells_per_thread": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lbm_set_graphs": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_set_wait_limit": (C.c_int, [C.c_void_p, C.c_uint]),
    "lbm_set_sweep_split": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_set_sweep_prefetch": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_set_remap_fused": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_set_momentum_stabilisation": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_set_sweep_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_get_sweep_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double),
                                       C.POINTER(C.c_longlong)]),
    "lbm_get_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong)]),
    "lbm_set_closure": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lbm_closure_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "lbm_mlp_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "lbm_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lbm_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_float, C.c_void_p]),
    "lbm_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_mlp_destroy": (C.c_int, [C.c_void_p]),
    "lbm_sbf_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lbm_sbf_set_fibres": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_sbf_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_sbf_destroy": (C.c_int, [C.c_void_p]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_status_string": (C.c_char_p, [C.c_int]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(st: int, ctx=None):
    if st != LBM_OK:
        lib = load()
        msg = lib.lbm_last_error(ctx).decode() if ctx else lib.lbm_status_string(st).decode()
        raise LBMError(st, msg or lib.lbm_status_string(st).decode())


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
# thin wrappers with the C names
# ---------------------------------------------------------------------------

def lbm_create(desc: lbm_grid_desc) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().lbm_create(C.byref(desc), C.byref(h)))
    return h


def lbm_create_batch(descs: Sequence[lbm_grid_desc]) -> C.c_void_p:
    arr = (lbm_grid_desc * len(descs))(*descs)
    h = C.c_void_p()
    _check(load().lbm_create_batch(arr, len(descs), C.byref(h)))
    return h


def lbm_set_particles(ctx, parts: Sequence[lbm_particle]):
    arr = (lbm_particle * max(len(parts), 1))(*parts)
    _check(load().lbm_set_particles(ctx, arr, len(parts)), ctx)


def lbm_step(ctx, nsteps: int):
    _check(load().lbm_step(ctx, nsteps), ctx)


def lbm_sync(ctx):
    _check(load().lbm_sync(ctx), ctx)


def lbm_get_forces(ctx, n: int, force: Optional[np.ndarray] = None, torque: Optional[np.ndarray] = None):
    F = force if force is not None else np.zeros((n, 3))
    M = torque if torque is not None else np.zeros((n, 3))
    _check(load().lbm_get_forces(ctx, _ptr(F), _ptr(M), n), ctx)
    return F, M


def lbm_get_wall_forces(ctx, cell: int = 0) -> np.ndarray:
    f = np.zeros(6)
    _check(load().lbm_get_wall_forces(ctx, cell, _ptr(f)), ctx)
    return f.reshape(2, 3)


def lbm_get_particles(ctx, n: int):
    arr = (lbm_particle * max(n, 1))()
    _check(load().lbm_get_particles(ctx, arr, n), ctx)
    return [arr[i] for i in range(n)]


def lbm_set_external(ctx, force: Optional[np.ndarray], torque: Optional[np.ndarray], n: int):
    _check(load().lbm_set_external(ctx, _ptr(force), _ptr(torque), n), ctx)


def lbm_get_fields(ctx, n: int, cell: int = 0, rho=True, u=True, flags=True, pid=True, pdfs=False):
    out = {}
    r = np.zeros(n) if rho else None
    uu = np.zeros((3, n)) if u else None
    fl = np.zeros(n, np.uint8) if flags else None
    pd = np.zeros(n, np.uint32) if pid else None
    pf = np.zeros((Q, n)) if pdfs else None
    _check(load().lbm_get_fields(ctx, cell, _ptr(r), _ptr(uu), _ptr(fl), _ptr(pd), _ptr(pf)), ctx)
    for k, v in (("rho", r), ("u", uu), ("flags", fl), ("pid", pd), ("pdfs", pf)):
        if v is not None:
            out[k] = v
    return out


def lbm_set_pdfs(ctx, pdfs: np.ndarray, cell: int = 0):
    pdfs = np.ascontiguousarray(pdfs, dtype=np.float64)
    _check(load().lbm_set_pdfs(ctx, cell, _ptr(pdfs)), ctx)


def lbm_get_links(ctx, cell: int = 0):
    lib = load()
    cnt = C.c_int(0)
    _check(lib.lbm_get_links(ctx, cell, None, None, None, 0, C.byref(cnt)), ctx)
    n = cnt.value
    idx = np.zeros(n, np.int32)
    q = np.zeros(n, np.int8)
    pid = np.zeros(n, np.uint32)
    _check(lib.lbm_get_links(ctx, cell, _ptr(idx), _ptr(q), _ptr(pid), n, C.byref(cnt)), ctx)
    return idx, q, pid


def lbm_get_info(ctx) -> lbm_info:
    info = lbm_info()
    _check(load().lbm_get_info(ctx, C.byref(info)), ctx)
    return info


def lbm_set_launch(ctx, block: int, grid: int = 0):
    _check(load().lbm_set_launch(ctx, block, grid), ctx)


def lbm_set_cells_per_thread(ctx, cpt: int):
    _check(load().lbm_set_cells_per_thread(ctx, cpt), ctx)


def lbm_autotune(ctx):
    b, g = C.c_int(0), C.c_int(0)
    _check(load().lbm_autotune(ctx, C.byref(b), C.byref(g)), ctx)
    return b.value, g.value


def lbm_set_sweep_split(ctx, enable: bool):
    _check(load().lbm_set_sweep_split(ctx, 1 if enable else 0), ctx)


# lbm_set_sweep_prefetch modes (include/lbm.h)
PREFETCH_OFF, PREFETCH_ALL, PREFETCH_EVEN, PREFETCH_ODD = 0, 1, 2, 3


def lbm_set_sweep_prefetch(ctx, mode):
    """mode: one of PREFETCH_OFF/ALL/EVEN/ODD; True / False stand for ALL / OFF."""
    if isinstance(mode, bool):
        mode = PREFETCH_ALL if mode else PREFETCH_OFF
    _check(load().lbm_set_sweep_prefetch(ctx, int(mode)), ctx)


def lbm_set_remap_fused(ctx, enable: bool):
    _check(load().lbm_set_remap_fused(ctx, 1 if enable else 0), ctx)


def lbm_set_momentum_stabilisation(ctx, enable: bool):
    _check(load().lbm_set_momentum_stabilisation(ctx, 1 if enable else 0), ctx)


def lbm_set_wait_limit(ctx, polls: int):
    _check(load().lbm_set_wait_limit(ctx, int(polls)), ctx)


def lbm_set_graphs(ctx, enable: bool):
    _check(load().lbm_set_graphs(ctx, int(bool(enable))), ctx)


def lbm_set_sweep_timing(ctx, enable: bool):
    _check(load().lbm_set_sweep_timing(ctx, int(bool(enable))), ctx)


def lbm_get_sweep_timing(ctx):
    ms, n = C.c_double(0), C.c_longlong(0)
    _check(load().lbm_get_sweep_timing(ctx, C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def lbm_get_launch_count(ctx) -> int:
    n = C.c_longlong(0)
    _check(load().lbm_get_launch_count(ctx, C.byref(n)), ctx)
    return n.value


def lbm_destroy(ctx):
    _check(load().lbm_destroy(ctx))


CLOSURE_IN, CLOSURE_OUT, CLOSURE_PARAMS = 86, 6, 14278


def lbm_set_closure(ctx, params_fp16: Optional[np.ndarray]):
    """Enable the learned closure with FP16 parameters (None disables)."""
    if params_fp16 is None:
        _check(load().lbm_set_closure(ctx, None, 0), ctx)
        return
    p = np.ascontiguousarray(params_fp16, dtype=np.float16)
    _check(load().lbm_set_closure(ctx, _ptr(p), p.nbytes), ctx)


def lbm_closure_features(ctx, n: int) -> np.ndarray:
    out = np.zeros((n, CLOSURE_IN), dtype=np.float32)
    _check(load().lbm_closure_features(ctx, _ptr(out), n), ctx)
    return out


def lbm_mlp_create(params: np.ndarray, stream_handle: int = 0) -> C.c_void_p:
    p = np.ascontiguousarray(params, dtype=np.float32)
    h = C.c_void_p()
    _check(load().lbm_mlp_create(_ptr(p), C.c_void_p(stream_handle), C.byref(h)))
    return h


def lbm_mlp_forward(m, x_ptr: int, y_ptr: int, n: int):
    _check(load().lbm_mlp_forward(m, C.c_void_p(x_ptr), C.c_void_p(y_ptr), n))


def lbm_mlp_grad(m, x_ptr: int, y_ptr: int, n: int, grad_ptr: int = 0) -> float:
    loss = np.zeros(1, dtype=np.float32)
    _check(load().lbm_mlp_grad(m, C.c_void_p(x_ptr), C.c_void_p(y_ptr), n, C.c_void_p(grad_ptr or None),
                               _ptr(loss)))
    return float(loss[0])


def lbm_mlp_train_step(m, x_ptr: int, y_ptr: int, n: int, lr: float, want_loss: bool = True):
    loss = np.zeros(1, dtype=np.float32)
    _check(load().lbm_mlp_train_step(m, C.c_void_p(x_ptr), C.c_void_p(y_ptr), n, C.c_float(lr),
                                     _ptr(loss) if want_loss else None))
    return float(loss[0]) if want_loss else None


def lbm_mlp_get_params(m):
    p32 = np.zeros(CLOSURE_PARAMS, dtype=np.float32)
    p16 = np.zeros(CLOSURE_PARAMS, dtype=np.float16)
    _check(load().lbm_mlp_get_params(m, _ptr(p32), _ptr(p16)))
    return p32, p16


def lbm_mlp_destroy(m):
    _check(load().lbm_mlp_destroy(m))


# --- slender-body formulation (include/lbm_sbf.h) --------------------------

class SlenderBodies:
    """Rigid straight fibres in unbounded Stokes flow (slender-body
    formulation) on the GPU: velocities for given forces and torques."""

    def __init__(self, centres, tangents, half_lengths, radii, mu: float, n_modes: int = 5, n_quad: int = 24,
                 stream=None):
        x = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
        self.M = len(x)
        h = C.c_void_p()
        _check(load().lbm_sbf_create(self.M, n_modes, n_quad, float(mu), stream, C.byref(h)))
        self.h = h
        self.set_fibres(x, tangents, half_lengths, radii)

    def set_fibres(self, centres, tangents, half_lengths, radii):
        M = self.M
        self._geo = [np.ascontiguousarray(centres, dtype=np.float64).reshape(M, 3),
                     np.ascontiguousarray(tangents, dtype=np.float64).reshape(M, 3),
                     np.ascontiguousarray(np.broadcast_to(half_lengths, (M,)), dtype=np.float64),
                     np.ascontiguousarray(np.broadcast_to(radii, (M,)), dtype=np.float64)]
        _check(load().lbm_sbf_set_fibres(self.h, *[_ptr(a) for a in self._geo]))

    def solve(self, forces, torques):
        F = np.ascontiguousarray(forces, dtype=np.float64).reshape(self.M, 3)
        T = np.ascontiguousarray(torques, dtype=np.float64).reshape(self.M, 3)
        xdot = np.zeros((self.M, 3))
        pdot = np.zeros((self.M, 3))
        _check(load().lbm_sbf_solve(self.h, _ptr(F), _ptr(T), _ptr(xdot), _ptr(pdot)))
        return xdot, pdot

    def close(self):
        if getattr(self, "h", None):
            load().lbm_sbf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# descriptors from lattice / particle records, torch-backed device memory
# ---------------------------------------------------------------------------

class TorchMemory:
    """Allocator callbacks that take device memory from torch's caching
    allocator on the given stream.  Keep the object alive with the context."""

    def __init__(self, stream, device: int = 0):
        import torch
        self._torch = torch
        self.stream = stream
        self.device = device
        self.live = {}

        def _alloc(nbytes, user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
            except Exception:
                return None
            self.live[p] = nbytes
            return p

        def _free(ptr, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_cb = ALLOC_FN(_alloc)
        self.free_cb = FREE_FN(_free)


def grid_desc(lat, prec: int = LBM_F32, stream_handle: int = 0,
              memory: Optional[TorchMemory] = None) -> lbm_grid_desc:
    d = lbm_grid_desc()
    d.nx, d.ny, d.nz = lat.nx, lat.ny, lat.nz
    d.tau, d.magic, d.rho0 = lat.tau, lat.magic, lat.rho0
    for a in range(3):
        d.periodic[a] = int(lat.periodic[a])
        d.wall_u_lo[a] = lat.wall_u_lo[a]
        d.wall_u_hi[a] = lat.wall_u_hi[a]
        d.body_force[a] = lat.body_force[a]
        d.free_slip[a] = int(getattr(lat, "free_slip", (0, 0, 0))[a])
    d.prec = prec
    d.cuda_stream = stream_handle or None
    if memory is not None:
        d.dev_alloc = memory.alloc_cb
        d.dev_free = memory.free_cb
    return d


def particle_struct(p) -> lbm_particle:
    s = lbm_particle()
    for a in range(3):
        s.pos[a] = p.pos[a]
        s.vel[a] = p.vel[a]
        s.omega[a] = p.omega[a]
        s.semi_axes[a] = p.semi_axes[a]
        s.ext_force[a] = p.ext_force[a]
        s.ext_torque[a] = p.ext_torque[a]
    for k in range(4):
        s.quat[k] = p.quat[k]
    s.density = p.density
    s.cell = p.cell
    s.fixed = p.fixed
    s.shape = getattr(p, "shape", 0)
    return s


def particle_array(parts: Sequence[lbm_particle]) -> np.ndarray:
    """Particle structs -> records (pos3 quat4 vel3 omega3 semi3 density extF3
    extM3 fixed cell shape), the layout the tests compare."""
    out = np.zeros((len(parts), 26))
    for i, s in enumerate(parts):
        out[i, 0:3] = list(s.pos)
        out[i, 3:7] = list(s.quat)
        out[i, 7:10] = list(s.vel)
        out[i, 10:13] = list(s.omega)
        out[i, 13:16] = list(s.semi_axes)
        out[i, 16] = s.density
        out[i, 17:20] = list(s.ext_force)
        out[i, 20:23] = list(s.ext_torque)
        out[i, 23] = s.fixed
        out[i, 24] = s.cell
        out[i, 25] = s.shape
    return out


class Simulation:
    """One context (a lattice or a batch of lattices) on a private torch
    stream, with torch-backed device memory."""

    def __init__(self, lattices, particles=(), prec: str | int = "f32", device: int = 0):
        import torch
        load()
        self.torch = torch
        torch.cuda.set_device(device)
        self.stream = torch.cuda.Stream(device=device)
        self.mem = TorchMemory(self.stream, device)
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else prec
        lats = lattices if isinstance(lattices, (list, tuple)) else [lattices]
        self.lattices = list(lats)
        self.descs = [grid_desc(l, self.prec, self.stream.cuda_stream, self.mem) for l in lats]
        if len(lats) == 1:
            self.h = lbm_create(self.descs[0])
        else:
            self.h = lbm_create_batch(self.descs)
        self.np = 0
        if len(particles):
            self.set_particles(particles)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, particles):
        structs = [particle_struct(p) for p in particles]
        lbm_set_particles(self.h, structs)
        self.np = len(structs)

    def set_momentum_stabilisation(self, enable: bool = True):
        lbm_set_momentum_stabilisation(self.h, enable)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def fields(self, cell: int = 0, pdfs: bool = True):
        lat = self.lattices[cell]
        f = lbm_get_fields(self.h, lat.ncells, cell, pdfs=pdfs)
        return f["rho"], f["u"], f["flags"], f["pid"], f.get("pdfs")

    def set_pdfs(self, pdfs, cell: int = 0):
        lbm_set_pdfs(self.h, pdfs, cell)

    def forces(self):
        return lbm_get_forces(self.h, self.np)

    def wall_forces(self, cell: int = 0):
        return lbm_get_wall_forces(self.h, cell)

    def particles(self) -> np.ndarray:
        return particle_array(lbm_get_particles(self.h, self.np))

    def links(self, cell: int = 0):
        return lbm_get_links(self.h, cell)

    def info(self) -> lbm_info:
        return lbm_get_info(self.h)

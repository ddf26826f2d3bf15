"""Failure detection of the C interface, made on the host or by bounded
device-side waits (nothing here faults, traps or hangs the GPU):

- LBM_ERR_OOM: a device allocator that refuses its k-th request, during
  lbm_create (every k) and during lbm_set_particles; nothing leaks, and a
  context whose body set could not be allocated stays usable without bodies;
- LBM_ERR_NUMERIC: a non-finite population written into one fluid cell next
  to a body through lbm_set_pdfs; the next step's force is non-finite, the
  synchronising call reports it and the context refuses further steps;
- LBM_ERR_TIMEOUT: the grid barriers of the fused re-mapping step given a
  poll limit of one, so that a waiting block gives up, sets the timeout bit
  and returns; reported the same way.
"""
import ctypes as C

import numpy as np
import pytest

from lbm_inputs import Particle, SplitMix64, quat_from_axis, shear_lattice, small_shear

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_06869_gb300 import _build, lbm as L
    _build.build()
    L.load()
    return L


class RefusingMemory:
    """Device memory from torch's caching allocator; request number
    `refuse_at` (0-based, counted from the last reset) returns NULL."""

    def __init__(self, lbm, stream):
        import torch
        self.stream = stream
        self.live = {}
        self.calls = 0
        self.refuse_at = None

        def _alloc(nbytes, user):
            k = self.calls
            self.calls += 1
            if self.refuse_at is not None and k == self.refuse_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream)
            self.live[p] = nbytes
            return p

        def _free(ptr, user):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_cb = lbm.ALLOC_FN(_alloc)
        self.free_cb = lbm.FREE_FN(_free)

    def reset(self, refuse_at=None):
        self.calls = 0
        self.refuse_at = refuse_at


def make(lbm, lat, mem, stream):
    d = lbm.grid_desc(lat, lbm.LBM_F32, stream.cuda_stream)
    d.dev_alloc = mem.alloc_cb
    d.dev_free = mem.free_cb
    return d


def test_oom_at_every_allocation_of_create(lbm):
    import torch
    stream = torch.cuda.Stream()
    mem = RefusingMemory(lbm, stream)
    lat = shear_lattice(20, 12, 10, 0.8, 0.01)
    mem.reset()
    h = lbm.lbm_create(make(lbm, lat, mem, stream))
    total = mem.calls
    lbm.lbm_destroy(h)
    assert total >= 10 and not mem.live
    for k in range(total):
        mem.reset(refuse_at=k)
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_create(make(lbm, lat, mem, stream))
        assert e.value.status == lbm.LBM_ERR_OOM, (k, e.value)
        assert not mem.live, f"refusing request {k} leaked {len(mem.live)} allocations"


def test_oom_in_set_particles_leaves_a_usable_context(lbm):
    import torch
    stream = torch.cuda.Stream()
    mem = RefusingMemory(lbm, stream)
    w = small_shear(seed=3, n=24, steps=10)
    lat = w.lattices[0]
    mem.reset()
    h = lbm.lbm_create(make(lbm, lat, mem, stream))
    parts = [lbm.particle_struct(p) for p in w.particles]
    for k in (0, 5, 24):
        mem.reset(refuse_at=k)
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_set_particles(h, parts)
        assert e.value.status == lbm.LBM_ERR_OOM
        # the lattice is mapped without bodies and steps
        f = lbm.lbm_get_fields(h, lat.ncells, 0, rho=False, u=True, flags=True, pid=True)
        assert not np.any(f["flags"] == lbm_flag_particle())
        lbm.lbm_step(h, 3)
        lbm.lbm_sync(h)
    # with the allocator working again the bodies map as in a fresh context
    mem.reset()
    lbm.lbm_set_particles(h, parts)
    f = lbm.lbm_get_fields(h, lat.ncells, 0, rho=False, u=False, flags=True, pid=True)
    ref = lbm.Simulation(lat, w.particles, prec="f32")
    _, _, fr, pr, _ = ref.fields(pdfs=False)
    assert np.array_equal(f["flags"], fr) and np.array_equal(f["pid"], pr)
    ref.close()
    lbm.lbm_destroy(h)
    assert not mem.live


def lbm_flag_particle():
    return 2


def test_nonfinite_population_is_reported_and_stops_the_context(lbm):
    w = small_shear(seed=5, n=24, steps=10)
    g = lbm.Simulation(w.lattices[0], w.particles, prec="f32")
    g.step(2)
    _, _, fl, pid, pdfs = g.fields()
    lat = w.lattices[0]
    # a fluid cell with a particle cell among its x neighbours
    part = (fl == 2).reshape(lat.nz, lat.ny, lat.nx)
    fluid = (fl == 0).reshape(lat.nz, lat.ny, lat.nx)
    cand = fluid & (np.roll(part, 1, axis=2) | np.roll(part, -1, axis=2))
    k, j, i = [int(v[0]) for v in np.nonzero(cand)]
    idx = i + lat.nx * (j + lat.ny * k)
    pdfs[:, idx] = np.nan
    g.set_pdfs(pdfs)
    g.step(1)
    with pytest.raises(lbm.LBMError) as e:
        g.sync()
    assert e.value.status == lbm.LBM_ERR_NUMERIC
    with pytest.raises(lbm.LBMError) as e:
        g.step(1)
    assert e.value.status == lbm.LBM_ERR_STATE
    g.close()


def test_barrier_wait_that_runs_out_is_reported(lbm):
    w = small_shear(seed=6, n=32, steps=10)
    g = lbm.Simulation(w.lattices[0], w.particles, prec="f32")
    lbm.lbm_set_remap_fused(g.h, True)
    info = lbm.lbm_get_info(g.h)
    if not info.remap_fused:
        g.close()
        pytest.skip("cooperative launches not available: no fused re-mapping step")
    g.step(4)
    g.sync()  # the default limit: no timeout
    lbm.lbm_set_wait_limit(g.h, 1)
    status = None
    for _ in range(20):
        try:
            g.step(1)
            g.sync()
        except lbm.LBMError as e:
            status = e.status
            break
    assert status == lbm.LBM_ERR_TIMEOUT
    with pytest.raises(lbm.LBMError) as e:
        g.step(1)
    assert e.value.status == lbm.LBM_ERR_STATE
    g.close()

"""The fused re-mapping step (rigid-body update and the uncover, claim,
fix-up and flags passes of Sec. 4.2-4.3 in one cooperative launch with grid
barriers) against the separate kernels.  The passes do the same arithmetic,
but the sweep's FP64 force sums come from atomics in no fixed order, so two
runs of either form agree to rounding only: flags and particle-id maps must be
identical, body states and fields equal to a few units of rounding of the
storage form.  The parity tests against the FP64 oracle run the separate
kernels (the default); these tests switch the fused form on explicitly.
"""
import numpy as np
import pytest

from lbm_inputs import batched_shear, fibre_suspension, small_shear

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


RTOL = {"f64": 1e-11, "f32": 1e-5, "f16": 1e-2}
# force and torque: sums of many link terms that largely cancel (the parity
# tests' force tolerances)
RTOL_FM = {"f64": 1e-9, "f32": 1e-4, "f16": 5e-2}


def state(sim, ncell):
    F, M = sim.forces()
    # force and torque on one scale (a centred body's force is round-off)
    out = {"particles": sim.particles(), "FM": np.concatenate([F.ravel(), M.ravel()])}
    for c in range(ncell):
        rho, u, fl, pid, _ = sim.fields(c)
        out[f"rho{c}"], out[f"u{c}"], out[f"flags{c}"], out[f"pid{c}"] = rho, u, fl, pid
    return out


def same(a, b, prec):
    for k in a:
        if k.startswith(("flags", "pid")):
            assert np.array_equal(a[k], b[k]), k
        else:
            scale = max(np.abs(b[k]).max(), 1e-300)
            err = np.abs(a[k] - b[k]).max() / scale
            assert err <= (RTOL_FM if k == "FM" else RTOL)[prec], (k, err)


def run(L, w, prec, fused, steps, graphs=True):
    s = L.Simulation(w.lattices, w.particles, prec=prec)
    L.lbm_set_remap_fused(s.h, fused)
    L.lbm_set_graphs(s.h, graphs)
    s.step(steps)
    info = s.info()
    st = state(s, len(w.lattices))
    s.close()
    return info, st


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_fused_matches_separate_single_body(lbm, prec):
    w = small_shear(seed=3, n=32)
    fi, a = run(lbm, w, prec, True, 60)
    si, b = run(lbm, w, prec, False, 60)
    assert fi.remap_fused == 1 and fi.remap_grid > 0, "cooperative launch not taken on this device"
    assert si.remap_fused == 0
    same(a, b, prec)


def test_fused_matches_separate_batched(lbm):
    w = batched_shear(seed=5, ncell=12, steps=40)
    fi, a = run(lbm, w, "f32", True, 40)
    _, b = run(lbm, w, "f32", False, 40)
    assert fi.remap_fused == 1
    same(a, b, "f32")


def test_fused_matches_separate_many_bodies_eager(lbm):
    """A fibre suspension with more region units than one resident wave: the
    fused kernel's blocks loop over units."""
    w = fibre_suspension(seed=2, nx=128, ny=96, nz=96, count=120, a=10.0, b=1.5)
    fi, a = run(lbm, w, "f32", True, 30, graphs=False)
    _, b = run(lbm, w, "f32", False, 30, graphs=False)
    assert fi.remap_fused == 1
    same(a, b, "f32")


def test_fused_launch_count(lbm):
    """One launch per re-mapping step in place of the rigid-body update and
    the re-mapping passes (uncover and claim in one pass for a single body,
    then fix-up and flags: four launches)."""
    w = small_shear(seed=3, n=32)
    counts = {}
    for fused in (True, False):
        s = lbm.Simulation(w.lattices, w.particles, prec="f32")
        lbm.lbm_set_remap_fused(s.h, fused)
        s.step(2)
        n0 = lbm.lbm_get_launch_count(s.h)
        s.step(10)
        counts[fused] = lbm.lbm_get_launch_count(s.h) - n0
        s.close()
    assert len(w.particles) == 1
    assert counts[False] - counts[True] == 10 * 3

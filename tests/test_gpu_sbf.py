"""The slender-body formulation on the GPU (`include/lbm_sbf.h`) against the
FP64 oracle (`oracle/sbf.py`, free space): one fibre, a pair, and five
fibres with random poses, forces and torques; argument errors."""
import numpy as np
import pytest

from oracle import sbf

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


def case(M, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-2.0, 2.0, (M, 3)) * np.array([1.0, 1.0, 1.0])
    x[:, 0] += 3.0 * np.arange(M)  # keep the fibres apart
    p = rng.normal(size=(M, 3))
    p /= np.linalg.norm(p, axis=1)[:, None]
    l = rng.uniform(0.8, 1.2, M)
    r = rng.uniform(0.04, 0.1, M)
    F = rng.normal(size=(M, 3))
    T = 0.3 * rng.normal(size=(M, 3))
    return x, p, l, r, F, T


@pytest.mark.parametrize("M,seed,n_modes,n_quad", [(1, 1, 5, 24), (2, 2, 5, 24), (5, 3, 6, 32)])
def test_velocities_match_the_oracle(lbm, M, seed, n_modes, n_quad):
    x, p, l, r, F, T = case(M, seed)
    mu = 0.8
    g = lbm.SlenderBodies(x, p, l, r, mu, n_modes=n_modes, n_quad=n_quad)
    vg, wg = g.solve(F, T)
    g.close()
    _, vo, wo = sbf.Fibres(x, p, l, r, mu, n_modes=n_modes, n_quad=n_quad).solve(F, T)
    assert np.allclose(vg, vo, rtol=1e-10, atol=1e-12 * np.abs(vo).max())
    assert np.allclose(wg, wo, rtol=1e-10, atol=1e-12 * np.abs(wo).max())


def test_argument_errors(lbm):
    with pytest.raises(lbm.LBMError):
        lbm.SlenderBodies([(0, 0, 0)], [(1, 0, 0)], [1.0], [1.5], 1.0)   # radius above the half length
    with pytest.raises(lbm.LBMError):
        lbm.SlenderBodies(np.zeros((65, 3)), np.tile([1.0, 0, 0], (65, 1)), 1.0, 0.1, 1.0)  # too many fibres
    with pytest.raises(lbm.LBMError):
        lbm.SlenderBodies([(0, 0, 0)], [(0, 0, 0)], [1.0], [0.1], 1.0)   # zero tangent

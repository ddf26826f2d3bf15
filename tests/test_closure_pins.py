"""Pins of the FP64 closure oracle (CPU only): each checks it against
something other than itself -- a special case that reduces to a matrix
product or a closed form, finite differences, the published Adam update,
exactness of trilinear interpolation on affine fields, and known rotations."""
import numpy as np
import pytest

from oracle import closure as cl
from lbm_inputs import SplitMix64


def rand_params(seed, scale=0.3):
    rng = SplitMix64(seed)
    return np.array([scale * (2 * rng.uniform() - 1) for _ in range(cl.N_PARAMS)])


def test_parameter_layout():
    assert cl.N_PARAMS == 64 * 86 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 6 * 64 + 6 == 14278
    theta = np.arange(cl.N_PARAMS, dtype=np.float64)
    L = cl.unpack(theta)
    assert L[0][0][0, 0] == 0 and L[0][0][0, 1] == 1 and L[0][0][1, 0] == 86   # W1 row-major [out][in]
    assert L[0][1][0] == 64 * 86                                                # b1 follows W1
    assert L[3][1][-1] == cl.N_PARAMS - 1                                       # b4 last
    np.testing.assert_array_equal(cl.pack(L), theta)


def test_forward_without_active_relu_is_the_matrix_product():
    # non-negative weights and inputs, zero biases: every ReLU passes its
    # input, so the network is the product W4 W3 W2 W1
    rng = np.random.default_rng(3)
    L = [(np.abs(rng.normal(size=(o, i))), np.zeros(o)) for o, i in cl.LAYERS]
    X = np.abs(rng.normal(size=(5, cl.N_IN)))
    out, _ = cl.forward(cl.pack(L), X)
    M = L[3][0] @ L[2][0] @ L[1][0] @ L[0][0]
    np.testing.assert_allclose(out, X @ M.T, rtol=1e-13)


def test_forward_dead_first_layer_leaves_the_biases():
    # W1 <= 0, b1 = 0 and x >= 0 switch the first hidden layer off; the output
    # is W4 relu(W3 relu(b2) + b3) + b4
    rng = np.random.default_rng(4)
    L = [(rng.normal(size=(o, i)), rng.normal(size=o)) for o, i in cl.LAYERS]
    L[0] = (-np.abs(L[0][0]), np.zeros(64))
    X = np.abs(rng.normal(size=(3, cl.N_IN)))
    out, _ = cl.forward(cl.pack(L), X)
    h2 = np.maximum(L[1][1], 0)
    h3 = np.maximum(L[2][0] @ h2 + L[2][1], 0)
    want = L[3][0] @ h3 + L[3][1]
    np.testing.assert_allclose(out, np.tile(want, (3, 1)), rtol=1e-13)


def test_forward_is_positively_homogeneous_without_biases():
    theta = rand_params(5)
    L = cl.unpack(theta.copy())
    for W, b in L:
        b[:] = 0.0
    theta0 = cl.pack(L)
    X = np.random.default_rng(5).normal(size=(4, cl.N_IN))
    o1, _ = cl.forward(theta0, X)
    o2, _ = cl.forward(theta0, 2.5 * X)
    np.testing.assert_allclose(o2, 2.5 * o1, rtol=1e-12, atol=1e-15)


def test_gradient_matches_central_differences():
    theta = rand_params(7)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(6, cl.N_IN))
    Y = rng.normal(size=(6, cl.N_OUT))
    _, g = cl.loss_and_grad(theta, X, Y)
    h = 1e-6
    idx = rng.choice(cl.N_PARAMS, size=60, replace=False)
    # include every block: first/last of each W and b
    k = 0
    for o, i in cl.LAYERS:
        idx = np.concatenate([idx, [k, k + o * i - 1, k + o * i, k + o * i + o - 1]])
        k += o * i + o
    for j in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (cl.loss_and_grad(tp, X, Y)[0] - cl.loss_and_grad(tm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(g[j])), (j, fd, g[j])


def test_loss_is_the_mean_squared_error():
    theta = rand_params(8)
    X = np.random.default_rng(8).normal(size=(4, cl.N_IN))
    out, _ = cl.forward(theta, X)
    loss, _ = cl.loss_and_grad(theta, X, out + 0.5)
    assert loss == pytest.approx(0.25, rel=1e-14)


def test_adam_first_two_steps_closed_form():
    # with zero moments the bias-corrected first step is g / (|g| + eps)
    g1 = np.array([0.3, -2.0, 1e-3, 0.0])
    opt = cl.Adam(4)
    th = opt.step(np.zeros(4), g1, lr=0.1)
    np.testing.assert_allclose(th, -0.1 * g1 / (np.abs(g1) + 1e-8), rtol=1e-12)
    g2 = np.array([0.1, 1.0, -1e-3, 2.0])
    th2 = opt.step(th, g2, lr=0.1)
    m = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.9 ** 2)
    v = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(th2, th - 0.1 * m / (np.sqrt(v) + 1e-8), rtol=1e-12)


def affine_field(dims, A, c):
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([i.ravel(), j.ravel(), k.ravel()])
    return A @ pts + c[:, None]


def test_trilinear_exact_on_affine_fields():
    dims = (7, 6, 5)
    rng = np.random.default_rng(11)
    A, c = rng.normal(size=(3, 3)), rng.normal(size=3)
    u3 = affine_field(dims, A, c)
    for _ in range(20):
        p = rng.uniform([0, 0, 0], [dims[0] - 1, dims[1] - 1, dims[2] - 1])
        np.testing.assert_allclose(cl.trilinear(u3, dims, (0, 0, 0), p), A @ p + c, rtol=1e-12, atol=1e-12)


def test_trilinear_periodic_wrap_and_clamp():
    dims = (4, 3, 3)
    u3 = np.zeros((3, 36))
    u3[0, 3] = 2.0   # cell (3, 0, 0)
    u3[0, 0] = 4.0   # cell (0, 0, 0)
    # halfway between cell 3 and its periodic image of cell 0 along x
    assert cl.trilinear(u3, dims, (1, 0, 0), (3.5, 0, 0))[0] == pytest.approx(3.0)
    # non-periodic: beyond the last cell the value is the last cell's
    assert cl.trilinear(u3, dims, (0, 0, 0), (3.5, 0, 0))[0] == pytest.approx(2.0)
    assert cl.trilinear(u3, dims, (0, 0, 0), (-0.7, 0, 0))[0] == pytest.approx(4.0)


def test_features_of_an_affine_flow_give_the_sample_points():
    # u = A x and a translating body: feature block s is R^T (A x_s - U) / V,
    # so with R = I it reveals the sample point x_s = x_C + (1.5a i, 1.5b j,
    # 1.5c k)
    dims = (40, 30, 30)
    A = np.diag([1.0, 2.0, 3.0])
    u3 = affine_field(dims, A, np.zeros(3))
    pos, semi, vel = np.array([20.0, 15.0, 15.0]), (6.0, 2.0, 2.0), np.array([0.5, 0.0, -0.25])
    gam = 0.01
    f = cl.features(u3, dims, (0, 0, 0), pos, (1, 0, 0, 0), vel, (0, 0, 0), semi, gam)
    V = gam * semi[0]
    s = 0
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                x = pos + np.array([9.0 * i, 3.0 * j, 3.0 * k])
                np.testing.assert_allclose(f[3 * s:3 * s + 3], (A @ x - vel) / V, rtol=1e-12)
                s += 1
    np.testing.assert_allclose(f[81:], [1, 0, 0, 3.0, 2.0])


def test_features_vanish_for_a_body_moving_rigidly_with_the_flow():
    # the rigid-body field u = U + Omega x (x - x_C) is affine, so its
    # trilinear interpolation is exact: a body translating with U and rotating
    # with Omega about x_C sees zero relative velocity at every sample point,
    # whatever its orientation
    dims = (40, 36, 38)
    pos = np.array([19.3, 17.6, 18.2])
    U, Om = np.array([0.01, -0.004, 0.007]), np.array([0.002, 0.003, -0.001])
    W = np.array([[0, -Om[2], Om[1]], [Om[2], 0, -Om[0]], [-Om[1], Om[0], 0]])
    u3 = affine_field(dims, W, U - W @ pos)
    q = np.array([0.8, 0.2, -0.4, 0.4])
    q /= np.linalg.norm(q)
    f = cl.features(u3, dims, (0, 0, 0), pos, q, U, Om, (6.0, 2.0, 1.5), 0.001)
    np.testing.assert_allclose(f[:81], 0.0, atol=1e-10)
    # and without the rotation term the same flow leaves Omega x r / V there
    f0 = cl.features(u3, dims, (0, 0, 0), pos, q, U, (0, 0, 0), (6.0, 2.0, 1.5), 0.001)
    assert np.abs(f0[:81]).max() > 1.0


def test_features_rotate_into_the_body_frame():
    # a uniform flow (1, 0, 0) seen by a body turned 90 degrees about z: its
    # x axis points along world y, so the flow has body components (0, -1, 0)
    dims = (20, 20, 20)
    u3 = np.zeros((3, 8000))
    u3[0] = 1.0
    q = (np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4))
    f = cl.features(u3, dims, (1, 1, 1), (10, 10, 10), q, (0, 0, 0), (0, 0, 0), (3, 1, 1), 0.0)
    for s in range(27):
        np.testing.assert_allclose(f[3 * s:3 * s + 3], [0, -1, 0], atol=1e-14)
    np.testing.assert_allclose(f[81:84], [0, 1, 0], atol=1e-15)


def test_closure_delta_scaling_and_frame():
    # zero weights, output bias e_0 / e_5: dF_body = mu*gam*a*b along x,
    # dM_body = mu*gam*a^2*b along z; a 90-degree turn about z maps body x to
    # world y and leaves z
    L = [(np.zeros((o, i)), np.zeros(o)) for o, i in cl.LAYERS]
    L[3][1][0] = 1.0
    L[3][1][5] = 2.0
    theta = cl.pack(L)
    tau, rho0, gam, semi = 0.8, 1.0, 3e-4, (12.0, 3.0, 3.0)
    mu = rho0 * (tau - 0.5) / 3.0
    q = (np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4))
    dF, dM = cl.closure_delta(theta, np.zeros(cl.N_IN), q, semi, tau, rho0, gam)
    np.testing.assert_allclose(dF, [0, mu * gam * 12 * 3, 0], atol=1e-18)
    np.testing.assert_allclose(dM, [0, 0, 2 * mu * gam * 144 * 3], atol=1e-18)


def test_wall_shear_rate_of_the_benchmark_channel():
    # walls at -0.02 / +0.02 on a 128-cell channel: 0.04 / 126
    assert cl.wall_shear_rate(128, -0.02, 0.02) == pytest.approx(3.1746e-4, rel=1e-4)

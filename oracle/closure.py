"""FP64 CPU reference of the learned force/torque closure.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the GPU
library and never imports it.

The paper's lattice Boltzmann model computes the hydrodynamic force and
torque on a body from the momentum exchanged across its boundary links
(Sec. 4.2, Eqs. TransferredMomentum, LBMhydrodynForce).  The learned closure
adds a correction (dF, dM) to them before the rigid-body update (Sec. 4.3),
predicted by a small multilayer perceptron from the flow around the body; the
paper itself has no such closure, so every definition below is a reading:

* Features (86 per body).  27 sample points in the body frame at offsets
  (1.5 a i, 1.5 b j, 1.5 c k), i, j, k in {-1, 0, 1}, point index
  s = 9 (i+1) + 3 (j+1) + (k+1), (a, b, c) the semi-axes; world point
  x_s = x_C + R o_s with R the rotation of the body's unit quaternion.  The
  velocity there is the trilinear interpolation of the cell-centred velocity
  field (cell (i, j, k) at the integer point (i, j, k); the field is the one
  the fields export reports: sum c f / rho0 + g/2 on fluid cells, zero on wall
  and particle cells); corner indices wrap on periodic axes and are clamped
  to [0, n-1] on the others.  Feature 3 s + d is component d of
  R^T (u(x_s) - U - Omega x (x_s - x_C)) / V: the fluid velocity relative to
  the body's rigid motion continued to the sample point (U the body's
  velocity, Omega its angular velocity), V = shear_rate * a (V = 1 when the
  shear rate is zero).  Features 81..83 are R's first column (the body's
  x axis in the world frame), 84 is a / b and 85 is b.
* Network: 86 -> 64 -> 64 -> 64 -> 6, ReLU after each hidden layer, linear
  output.  Parameters in one flat vector: W1 (64 x 86, row-major, [out][in]),
  b1 (64), W2 (64 x 64), b2, W3 (64 x 64), b3, W4 (6 x 64), b4 (6):
  14,278 values.
* Outputs: o[0:3] is dF in the body frame in units of mu * shear_rate * a * b,
  o[3:6] is dM in the body frame in units of mu * shear_rate * a^2 * b, with
  mu = rho0 (tau - 1/2) / 3; the world-frame correction is R dF, R dM.
* Training: loss = mean over the batch and the 6 outputs of (o - y)^2; Adam
  (Kingma & Ba, 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 on the
  parameters.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 86, 64, 6
LAYERS = ((N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (N_OUT, N_HID))
N_PARAMS = sum(o * i + o for o, i in LAYERS)  # 14,278


def unpack(theta):
    """Flat parameter vector -> [(W, b), ...] (views, FP64)."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    out, k = [], 0
    for o, i in LAYERS:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers]).astype(np.float64)


def forward(theta, X):
    """Network outputs for the rows of X (n x 86) and the activations."""
    X = np.asarray(X, dtype=np.float64)
    acts = [X]
    h = X
    L = unpack(theta)
    for li, (W, b) in enumerate(L):
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if li < len(L) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grad(theta, X, Y):
    """Mean squared error and its gradient with respect to theta, by
    back-propagation through the layers in reverse order."""
    out, acts = forward(theta, X)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[0]
    diff = out - Y
    loss = float(np.mean(diff * diff))
    L = unpack(theta)
    grads = [None] * len(L)
    d = 2.0 * diff / (n * N_OUT)          # dL/d(output)
    for li in range(len(L) - 1, -1, -1):
        W, _ = L[li]
        h_in = acts[li]
        grads[li] = (d.T @ h_in, d.sum(axis=0))
        if li > 0:
            d = (d @ W) * (acts[li] > 0.0)  # through the ReLU of the layer below
    return loss, pack(grads)


class Adam:
    """Adam optimiser state over a flat parameter vector."""

    def __init__(self, n, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.b1, self.b2, self.eps = beta1, beta2, eps

    def step(self, theta, grad, lr):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        mhat = self.m / (1.0 - self.b1 ** self.t)
        vhat = self.v / (1.0 - self.b2 ** self.t)
        return theta - lr * mhat / (np.sqrt(vhat) + self.eps)


def quat_rotation(q):
    """Rotation matrix (body -> world) of the quaternion (w, x, y, z)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def trilinear(u3, dims, periodic, point):
    """Trilinear interpolation of the cell-centred field u3 (3 x n, x fastest)
    at a world point."""
    nx, ny, nz = dims
    n = np.array(dims)
    p = np.asarray(point, dtype=np.float64)
    i0 = np.floor(p).astype(int)
    w1 = p - i0
    out = np.zeros(3)
    for c in range(8):
        off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
        idx = i0 + off
        wgt = 1.0
        for a in range(3):
            wgt *= w1[a] if off[a] else 1.0 - w1[a]
            if periodic[a]:
                idx[a] %= n[a]
            else:
                idx[a] = min(max(idx[a], 0), n[a] - 1)
        lin = idx[0] + nx * (idx[1] + ny * idx[2])
        out += wgt * u3[:, lin]
    return out


def sample_offsets(semi):
    a, b, c = semi
    offs = []
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                offs.append((1.5 * a * i, 1.5 * b * j, 1.5 * c * k))
    return np.array(offs)


def features(u3, dims, periodic, pos, quat, vel, omega, semi, shear_rate):
    """The 86 closure inputs of one body (see the module docstring)."""
    R = quat_rotation(quat)
    a, b = semi[0], semi[1]
    V = shear_rate * a if shear_rate > 0 else 1.0
    f = np.zeros(N_IN)
    for s, o in enumerate(sample_offsets(semi)):
        r = R @ o
        x = np.asarray(pos) + r
        u = trilinear(u3, dims, periodic, x)
        rigid = np.asarray(vel) + np.cross(np.asarray(omega), r)
        f[3 * s:3 * s + 3] = R.T @ (u - rigid) / V
    f[81:84] = R[:, 0]
    f[84] = a / b
    f[85] = b
    return f


def closure_delta(theta, feats, quat, semi, tau, rho0, shear_rate):
    """World-frame (dF, dM) of one body from its features."""
    out, _ = forward(theta, np.asarray(feats)[None, :])
    o = out[0]
    R = quat_rotation(quat)
    a, b = semi[0], semi[1]
    mu = rho0 * (tau - 0.5) / 3.0
    fs = mu * shear_rate * a * b
    ms = mu * shear_rate * a * a * b
    return R @ (o[:3] * fs), R @ (o[3:] * ms)


def wall_shear_rate(ny, wall_u_lo_x, wall_u_hi_x):
    """Shear rate of the channel between the moving walls y = 0 and y = ny-1
    (half-way bounce-back puts the walls at y = 0.5 and ny - 1.5)."""
    return abs(wall_u_hi_x - wall_u_lo_x) / (ny - 2.0)

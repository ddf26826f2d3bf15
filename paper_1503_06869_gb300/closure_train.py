"""Training data, training and evaluation of the learned force/torque closure.

A sample is one fixed spheroid in simple shear at a seeded orientation,
simulated twice to the same physical time: on the coarse lattice (minor
semi-axis b, the resolution the closure is meant for) and on a lattice four
times finer (diffusive scaling: dx / 4, dt / 16, same tau, so the wall speed
is a quarter and the run 16 times longer).  Features are those of the coarse
run (``lbm_closure_features``); the target is the difference of the two runs'
hydrodynamic force and torque in the body frame, in the closure's units
F / (mu gamma a b) and M / (mu gamma a^2 b).  The network is trained on the GPU
(``lbm_mlp_*``) and scored on held-out orientations: the error of the coarse
force/torque against the fine one without and with the predicted correction.

    python -m paper_1503_06869_gb300.closure_train --samples 40 --out closure.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from lbm_inputs import Particle, SplitMix64, quat_from_axis, shear_lattice  # noqa: E402
from paper_1503_06869_gb300 import lbm  # noqa: E402

_W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
_CX = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0], dtype=float)


def couette_pdfs(lat):
    """Equilibrium populations of the Couette profile between the half-way
    walls at y = 0.5 and y = ny - 1.5."""
    y = np.arange(lat.ny, dtype=float)
    ux = lat.wall_u_lo[0] + (lat.wall_u_hi[0] - lat.wall_u_lo[0]) * (y - 0.5) / (lat.ny - 2.0)
    cu = np.outer(_CX, ux)
    feq = _W[:, None] * lat.rho0 * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * ux[None, :] ** 2)
    n = lat.nx * lat.ny * lat.nz
    return np.ascontiguousarray(feq[:, (np.arange(n) // lat.nx) % lat.ny])


def rotation(q):
    w, x, y, z = np.asarray(q, dtype=float) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def run_case(box, a, b, uw, tau, steps, quat, features=False):
    """Fixed spheroid at the box centre in Couette flow: force and torque of
    the last step in the body frame, in units mu gamma a b and mu gamma a^2 b,
    and (optionally) the closure features."""
    lat = shear_lattice(box[0], box[1], box[2], tau, uw)
    pos = ((box[0] - 1) / 2.0, (box[1] - 1) / 2.0, (box[2] - 1) / 2.0)
    p = Particle(pos=pos, quat=quat, semi_axes=(a, b, b), fixed=1)
    sim = lbm.Simulation([lat], [p], prec="f32")
    try:
        sim.set_pdfs(couette_pdfs(lat))
        sim.step(steps)
        F, M = sim.forces()
        feat = lbm.lbm_closure_features(sim.h, 1)[0] if features else None
    finally:
        sim.close()
    mu = lat.rho0 * (tau - 0.5) / 3.0
    gamma = abs(2 * uw) / (box[1] - 2.0)
    R = rotation(quat)
    Fb = R.T @ F[0] / (mu * gamma * a * b)
    Mb = R.T @ M[0] / (mu * gamma * a * a * b)
    return np.concatenate([Fb, Mb]), feat


def make_samples(n, seed=1, coarse_box=(48, 40, 48), a=15.0, b=1.5, uw=0.02, tau=0.8, coarse_steps=1000,
                 scale=4, log=print):
    """n (features, target, coarse, fine) samples at seeded orientations."""
    rng = SplitMix64(seed)
    fine_box = (scale * coarse_box[0], scale * (coarse_box[1] - 2) + 2, scale * coarse_box[2])
    X, Y, C, Fn = [], [], [], []
    for i in range(n):
        q = quat_from_axis(rng.unit_vector())
        yc, feat = run_case(coarse_box, a, b, uw, tau, coarse_steps, q, features=True)
        yf, _ = run_case(fine_box, scale * a, scale * b, uw / scale, tau, coarse_steps * scale * scale, q)
        X.append(feat)
        Y.append(yf - yc)
        C.append(yc)
        Fn.append(yf)
        log(f"sample {i}: coarse {np.round(yc, 4).tolist()} fine {np.round(yf, 4).tolist()}")
    return np.array(X), np.array(Y), np.array(C), np.array(Fn)


def init_params(seed):
    """He-normal weights, zero biases, in the flat layout of lbm.h."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in ((64, 86), (64, 64), (64, 64), (6, 64)):
        parts.append(rng.normal(size=o * i) * math.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def train(X, Y, steps=2000, lr=1e-3, seed=0, Xv=None, Yv=None, every=50):
    """Full-batch Adam on the GPU; returns FP32 and FP16 parameters and the
    loss history.  With a validation set (Xv, Yv), the parameters returned
    are those of the lowest validation loss, checked every `every` steps
    (early stopping)."""
    import torch
    m = lbm.lbm_mlp_create(init_params(seed))
    try:
        x = torch.tensor(np.ascontiguousarray(X, dtype=np.float32), device="cuda")
        y = torch.tensor(np.ascontiguousarray(Y, dtype=np.float32), device="cuda")
        if Xv is not None:
            xv = torch.tensor(np.ascontiguousarray(Xv, dtype=np.float32), device="cuda")
            yv = torch.tensor(np.ascontiguousarray(Yv, dtype=np.float32), device="cuda")
        hist, best, best_p = [], math.inf, None
        for s in range(steps):
            loss = lbm.lbm_mlp_train_step(m, x.data_ptr(), y.data_ptr(), len(X), lr, want_loss=(s % every == 0))
            if loss is not None:
                hist.append(loss)
            if Xv is not None and (s + 1) % every == 0:
                vl = lbm.lbm_mlp_grad(m, xv.data_ptr(), yv.data_ptr(), len(Xv))
                if vl < best:
                    best, best_p = vl, lbm.lbm_mlp_get_params(m)
        p32, p16 = best_p if best_p is not None else lbm.lbm_mlp_get_params(m)
    finally:
        lbm.lbm_mlp_destroy(m)
    return p32, p16, hist


def predict(p32, X):
    import torch
    m = lbm.lbm_mlp_create(p32)
    try:
        x = torch.tensor(np.ascontiguousarray(X, dtype=np.float32), device="cuda")
        y = torch.zeros((len(X), 6), device="cuda")
        lbm.lbm_mlp_forward(m, x.data_ptr(), y.data_ptr(), len(X))
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64)
    finally:
        lbm.lbm_mlp_destroy(m)


def evaluate(C, Fn, pred):
    """RMS over held-out samples of the coarse error against the fine run,
    force and torque parts, without and with the predicted correction."""
    def rms(e):
        return float(np.sqrt(np.mean(np.sum(e * e, axis=1))))
    return {"force_rms_without": rms(C[:, :3] - Fn[:, :3]), "force_rms_with": rms(C[:, :3] + pred[:, :3] - Fn[:, :3]),
            "torque_rms_without": rms(C[:, 3:] - Fn[:, 3:]), "torque_rms_with": rms(C[:, 3:] + pred[:, 3:] - Fn[:, 3:])}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=160)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--val", type=int, default=24)
    ap.add_argument("--coarse-steps", type=int, default=1000)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--data", default="", help="reuse the samples of an earlier --out file")
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    lbm.load()
    if args.data:
        d = np.load(args.data)
        X, Y, C, Fn = d["X"], d["Y"], d["coarse"], d["fine"]
    else:
        X, Y, C, Fn = make_samples(args.samples, coarse_steps=args.coarse_steps, log=lambda s: print(s, flush=True))
    n = len(X)
    ntr = n - args.test - args.val
    p32, p16, hist = train(X[:ntr], Y[:ntr], steps=args.train_steps, lr=args.lr,
                           Xv=X[ntr:n - args.test], Yv=Y[ntr:n - args.test])
    te = slice(n - args.test, n)
    res = {"samples": n, "train": ntr, "validation": args.val, "held_out": args.test,
           "train_loss_first_last": [hist[0], hist[-1]], **evaluate(C[te], Fn[te], predict(p32, X[te]))}
    print(json.dumps(res), flush=True)
    if args.out:
        np.savez(args.out, X=X, Y=Y, coarse=C, fine=Fn, params32=p32, params16=p16)
    return res


if __name__ == "__main__":
    main()

"""Training data, training and evaluation of the learned force/torque closure.

Two data sets, both from paired runs of the method itself at two resolutions
(diffusive scaling: dx / s, dt / s^2, same tau, wall speed / s, s = 4 for the
b = 1.5 / b = 6 pairs):

* moving bodies (``paired_moving``, the closure's training set): batches of
  independent shear cells, one prolate spheroid each, rotating at a seeded
  angular velocity perpendicular to its axis (|Omega| up to 1.5 gamma) about
  the centre of the channel; the body is made so heavy (density 1e12) that
  the flow cannot change its motion, so the coarse and the fine body follow
  the same prescribed motion exactly (a rotation about a fixed axis composes
  exactly over the s^2 fine steps of one coarse step).  After a transient,
  every `spacing` coarse steps one sample: the features of the coarse run at
  the start of a window of `window` coarse steps, and the force and torque of
  both runs averaged over that window (the matched s^2 window fine steps);
* fixed bodies (``make_samples``): one fixed spheroid per run at a seeded
  orientation, force and torque of the last step.

The target is the difference fine - coarse of the body-frame force and torque
in the closure's units F / (mu gamma a b) and M / (mu gamma a^2 b) (equal
physical loads have equal values at both resolutions).  The network is
trained on the GPU (``lbm_mlp_*``) and scored on held-out bodies: the error
of the coarse force/torque against the fine one without the closure, with a
single fitted scale factor per part (fine ~ c coarse), and with the network.

    python -m paper_1503_06869_gb300.closure_train --moving --bodies 200 --samples-per-body 100
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


HEAVY = 1e12  # body density of the prescribed-motion runs: hydrodynamic loads do not move the body


def _channel_centre(box):
    return ((box[0] - 1) / 2.0, (box[1] - 1) / 2.0, (box[2] - 1) / 2.0)


def _body_frame_nd(F, M, quats, mu, gamma, a, b):
    """World-frame F, M (n x 3) -> body-frame, nondimensional (n x 6)."""
    out = np.zeros((len(F), 6))
    for i in range(len(F)):
        R = rotation(quats[i])
        out[i, :3] = R.T @ F[i] / (mu * gamma * a * b)
        out[i, 3:] = R.T @ M[i] / (mu * gamma * a * a * b)
    return out


def paired_moving(nbody, seed=11, coarse_box=(48, 40, 48), a=15.0, b=1.5, uw=0.02, tau=0.8, scale=4,
                  transient=400, samples=100, spacing=12, window=4, max_spin=1.5, fine_prec="f16",
                  log=print):
    """Paired coarse/fine runs of `nbody` rotating spheroids (one per shear
    cell, all cells of a resolution in one batch).  Returns features X (n x
    86), targets Y = fine - coarse (n x 6), the coarse and fine loads C, Fn
    (n x 6, body frame, closure units) and the body index of every sample."""
    rng = SplitMix64(seed)
    gamma = abs(2 * uw) / (coarse_box[1] - 2.0)
    fine_box = (scale * coarse_box[0], scale * (coarse_box[1] - 2) + 2, scale * coarse_box[2])
    lc = shear_lattice(coarse_box[0], coarse_box[1], coarse_box[2], tau, uw)
    lf = shear_lattice(fine_box[0], fine_box[1], fine_box[2], tau, uw / scale)
    pc, pf = [], []
    for i in range(nbody):
        t = np.array(rng.unit_vector())
        v = np.array(rng.unit_vector())
        n = v - np.dot(v, t) * t
        n /= np.linalg.norm(n)
        w = rng.uniform_range(-max_spin, max_spin) * gamma
        q = quat_from_axis(tuple(t))
        pc.append(Particle(pos=_channel_centre(coarse_box), quat=q, semi_axes=(a, b, b), density=HEAVY,
                           omega=tuple(w * n), cell=i))
        pf.append(Particle(pos=_channel_centre(fine_box), quat=q, semi_axes=(scale * a, scale * b, scale * b),
                           density=HEAVY, omega=tuple(w * n / scale ** 2), cell=i))
    sims = []
    try:
        sc = lbm.Simulation([lc] * nbody, pc, prec="f32")
        sims.append(sc)
        sf = lbm.Simulation([lf] * nbody, pf, prec=fine_prec)
        sims.append(sf)
        for c in range(nbody):
            sc.set_pdfs(couette_pdfs(lc), c)
            sf.set_pdfs(couette_pdfs(lf), c)
        lbm.lbm_autotune(sc.h)
        lbm.lbm_autotune(sf.h)
        sc.step(transient)
        sf.step(transient * scale * scale)
        mu = lc.rho0 * (tau - 0.5) / 3.0
        X, C, Fn, body = [], [], [], []
        for k in range(samples):
            sc.step(spacing - window)
            sf.step((spacing - window) * scale * scale)
            X.append(lbm.lbm_closure_features(sc.h, nbody))
            quats = sc.particles()[:, 3:7]
            Fc = np.zeros((nbody, 3)); Mc = np.zeros((nbody, 3))
            Ff = np.zeros((nbody, 3)); Mf = np.zeros((nbody, 3))
            for _ in range(window):
                sc.step(1)
                F, M = sc.forces()
                Fc += F; Mc += M
            for _ in range(window * scale * scale):
                sf.step(1)
                F, M = sf.forces()
                Ff += F; Mf += M
            nf = window * scale * scale
            C.append(_body_frame_nd(Fc / window, Mc / window, quats, mu, gamma, a, b))
            # fine loads in coarse closure units: equal physical forces have
            # equal lattice values under diffusive scaling, torques scale by s
            Fn.append(_body_frame_nd(Ff / nf, Mf / nf / scale, quats, mu, gamma, a, b))
            body.append(np.arange(nbody))
            if k % 10 == 0:
                log(f"sample round {k}: coarse torque rms {np.sqrt(np.mean(C[-1][:, 3:] ** 2)):.3f}, "
                    f"fine {np.sqrt(np.mean(Fn[-1][:, 3:] ** 2)):.3f}")
    finally:
        for sim in sims:
            sim.close()
    X = np.concatenate(X)
    C = np.concatenate(C)
    Fn = np.concatenate(Fn)
    return X, Fn - C, C, Fn, np.concatenate(body)


def fit_scale(C, Fn):
    """Least-squares factors c_F, c_M with Fn ~ c C, separately for the force
    and the torque part (the one-parameter-per-part baseline)."""
    cF = float(np.sum(C[:, :3] * Fn[:, :3]) / max(np.sum(C[:, :3] ** 2), 1e-300))
    cM = float(np.sum(C[:, 3:] * Fn[:, 3:]) / max(np.sum(C[:, 3:] ** 2), 1e-300))
    return cF, cM


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


def evaluate(C, Fn, pred, scale=None):
    """RMS over held-out samples of the coarse error against the fine run,
    force and torque parts, without and with the predicted correction (and,
    given the factors (c_F, c_M), with the coarse loads rescaled)."""
    def rms(e):
        return float(np.sqrt(np.mean(np.sum(e * e, axis=1))))
    res = {"force_rms_without": rms(C[:, :3] - Fn[:, :3]), "force_rms_with": rms(C[:, :3] + pred[:, :3] - Fn[:, :3]),
           "torque_rms_without": rms(C[:, 3:] - Fn[:, 3:]), "torque_rms_with": rms(C[:, 3:] + pred[:, 3:] - Fn[:, 3:]),
           "force_rms_fine": rms(Fn[:, :3]), "torque_rms_fine": rms(Fn[:, 3:])}
    if scale is not None:
        res["force_rms_scaled"] = rms(scale[0] * C[:, :3] - Fn[:, :3])
        res["torque_rms_scaled"] = rms(scale[1] * C[:, 3:] - Fn[:, 3:])
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--moving", action="store_true", help="paired runs of rotating bodies (the training set)")
    ap.add_argument("--bodies", type=int, default=200)
    ap.add_argument("--held-out-bodies", type=int, default=20)
    ap.add_argument("--val-bodies", type=int, default=10)
    ap.add_argument("--samples-per-body", type=int, default=100)
    ap.add_argument("--batch", type=int, default=100, help="bodies per paired batch run")
    ap.add_argument("--samples", type=int, default=160, help="fixed bodies: number of runs")
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--val", type=int, default=24)
    ap.add_argument("--coarse-steps", type=int, default=1000)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--data", default="", help="reuse the samples of an earlier --out file")
    ap.add_argument("--out", default="")
    ap.add_argument("--params-out", default="", help="write the trained FP16 parameters (.npy)")
    ap.add_argument("--eval-out", default="", help="write the held-out evaluation (.json)")
    args = ap.parse_args(argv)
    lbm.load()
    log = lambda m: print(m, flush=True)  # noqa: E731
    if args.data:
        d = np.load(args.data)
        X, Y, C, Fn = d["X"], d["Y"], d["coarse"], d["fine"]
        body = d["body"] if "body" in d else None
    elif args.moving:
        parts = []
        done = 0
        while done < args.bodies:
            nb = min(args.batch, args.bodies - done)
            Xb, Yb, Cb, Fb, bb = paired_moving(nb, seed=1000 + done, samples=args.samples_per_body, log=log)
            parts.append((Xb, Yb, Cb, Fb, bb + done))
            done += nb
        X, Y, C, Fn, body = (np.concatenate([p[i] for p in parts]) for i in range(5))
    else:
        X, Y, C, Fn = make_samples(args.samples, coarse_steps=args.coarse_steps, log=log)
        body = None
    if body is not None:
        # split by body: held-out and validation bodies are never trained on
        nbodies = int(body.max()) + 1
        te = body >= nbodies - args.held_out_bodies
        va = (body >= nbodies - args.held_out_bodies - args.val_bodies) & ~te
        tr = ~te & ~va
    else:
        n = len(X)
        idx = np.arange(n)
        te = idx >= n - args.test
        va = (idx >= n - args.test - args.val) & ~te
        tr = ~te & ~va
    p32, p16, hist = train(X[tr], Y[tr], steps=args.train_steps, lr=args.lr, Xv=X[va], Yv=Y[va])
    cF, cM = fit_scale(C[tr], Fn[tr])
    res = {"samples": int(len(X)), "train": int(tr.sum()), "validation": int(va.sum()), "held_out": int(te.sum()),
           "train_loss_first_last": [hist[0], hist[-1]], "scale_factors": [cF, cM],
           **evaluate(C[te], Fn[te], predict(p32, X[te]), scale=(cF, cM))}
    print(json.dumps(res), flush=True)
    if args.out:
        np.savez(args.out, X=X, Y=Y, coarse=C, fine=Fn, params32=p32, params16=p16,
                 **({"body": body} if body is not None else {}))
    if args.params_out:
        np.save(args.params_out, p16)
    if args.eval_out:
        with open(args.eval_out, "w") as fh:
            json.dump(res, fh, indent=1)
    return res


if __name__ == "__main__":
    main()

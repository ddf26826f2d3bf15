"""Training data, training and evaluation of the learned force/torque closure.

Two data sets, both from paired runs of the method itself at two resolutions
(diffusive scaling: dx / s, dt / s^2, same tau, wall speed / s, s = 4 for the
b = 1.5 / b = 6 pairs):

* moving bodies (``paired_moving``, the closure's training set): batches of
  independent shear cells, one prolate spheroid each, rotating at a seeded
  angular velocity perpendicular to its axis (|Omega| up to 1.5 gamma) and
  translating with a seeded slip parallel to the walls (up to 0.5 gamma a)
  from the middle of the channel; the body is made so heavy (density 1e12)
  that the flow cannot change its motion, so the coarse and the fine body
  follow the same prescribed motion exactly (a rotation about a fixed axis and
  a constant translation compose exactly over the s^2 fine steps of one
  coarse step).  After a transient,
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
                  transient=400, samples=100, spacing=12, window=4, max_spin=1.5, max_slip=0.5,
                  fine_prec="f16", log=print):
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
        # slip against the flow, parallel to the walls (the centre stays on
        # the channel's middle plane, where the flow is at rest)
        phi = rng.uniform_range(0.0, 2.0 * math.pi)
        us = rng.uniform_range(0.0, max_slip) * gamma * a
        U = np.array([us * math.cos(phi), 0.0, us * math.sin(phi)])
        q = quat_from_axis(tuple(t))
        pc.append(Particle(pos=_channel_centre(coarse_box), quat=q, semi_axes=(a, b, b), density=HEAVY,
                           vel=tuple(U), omega=tuple(w * n), cell=i))
        pf.append(Particle(pos=_channel_centre(fine_box), quat=q, semi_axes=(scale * a, scale * b, scale * b),
                           density=HEAVY, vel=tuple(U / scale), omega=tuple(w * n / scale ** 2), cell=i))
    sims = []
    try:
        sc = lbm.Simulation([lc] * nbody, pc, prec="f32")
        sims.append(sc)
        sf = lbm.Simulation([lf] * nbody, pf, prec=fine_prec)
        sims.append(sf)
        pdc, pdf = couette_pdfs(lc), couette_pdfs(lf)
        for c in range(nbody):
            sc.set_pdfs(pdc, c)
            sf.set_pdfs(pdf, c)
        del pdc, pdf
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


def fluctuation(C, Fn, body, scale):
    """Step-to-step fluctuation of the rescaled coarse error: the RMS of the
    difference between consecutive samples of the same body, over sqrt 2,
    per part.  Consecutive samples are a few steps apart, so their smooth
    parts agree; what remains is the staircase fluctuation of the coarse
    momentum exchange, which no function of the (smooth) flow features can
    predict: a floor for the error of any such closure."""
    out = []
    for sl, c in ((slice(0, 3), scale[0]), (slice(3, 6), scale[1])):
        R = c * C[:, sl] - Fn[:, sl]
        d = [np.diff(R[body == b], axis=0) for b in np.unique(body)]
        d = np.concatenate([x for x in d if len(x)])
        out.append(float(np.sqrt(np.mean(np.sum(d * d, axis=1)) / 2.0)))
    return out


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


LAYERS = ((64, 86), (64, 64), (64, 64), (6, 64))  # (out, in) of the four layers, lbm.h layout


def split_params(p):
    """Flat parameter vector -> [(W, b)] per layer (views)."""
    out, o = [], 0
    for n_out, n_in in LAYERS:
        W = p[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        b = p[o:o + n_out]
        o += n_out
        out.append((W, b))
    return out


def fold_standardisation(p32, mX, sX, sY):
    """Parameters trained on standardised data ((X - mX) / sX -> Y / sY) ->
    parameters of the same network on raw features and targets: the input
    scaling folds into the first layer, the output scaling into the last."""
    p = np.array(p32, dtype=np.float64)
    (W1, b1), _, _, (W4, b4) = split_params(p)
    b1 -= W1 @ (mX / sX)
    W1 /= sX[None, :]
    W4 *= sY[:, None]
    b4 *= sY
    return p.astype(np.float32)


def standardisation(X, Y):
    """Feature means and scales (constant features: mean 0, scale 1) and
    target scales (per output)."""
    mX = X.mean(axis=0)
    sX = X.std(axis=0)
    const = sX < 1e-6
    mX[const] = 0.0
    sX[const] = 1.0
    # a floor on the scales keeps the folded first layer (W / sX) well inside
    # the FP16 range
    if (~const).any():
        sX[~const] = np.maximum(sX[~const], 0.05 * np.median(sX[~const]))
    sY = np.sqrt((Y ** 2).mean(axis=0))
    sY[sY < 1e-6] = 1.0
    return mX, sX, sY


def train(X, Y, steps=2000, lr=1e-3, seed=0, Xv=None, Yv=None, every=50, standardise=True):
    """Full-batch Adam on the GPU; returns FP32 and FP16 parameters (for raw
    features and targets) and the loss history.  With standardise, the
    network is trained on standardised features and targets and the scales
    are folded into the first and last layers afterwards.  With a validation
    set (Xv, Yv), the parameters returned are those of the lowest validation
    loss, checked every `every` steps (early stopping)."""
    import torch
    if standardise:
        mX, sX, sY = standardisation(X, Y)
    else:
        mX, sX, sY = np.zeros(X.shape[1]), np.ones(X.shape[1]), np.ones(Y.shape[1])
    m = lbm.lbm_mlp_create(init_params(seed))
    try:
        x = torch.tensor(np.ascontiguousarray((X - mX) / sX, dtype=np.float32), device="cuda")
        y = torch.tensor(np.ascontiguousarray(Y / sY, dtype=np.float32), device="cuda")
        if Xv is not None:
            xv = torch.tensor(np.ascontiguousarray((Xv - mX) / sX, dtype=np.float32), device="cuda")
            yv = torch.tensor(np.ascontiguousarray(Yv / sY, dtype=np.float32), device="cuda")
        hist, best, best_p = [], math.inf, None
        for s in range(steps):
            loss = lbm.lbm_mlp_train_step(m, x.data_ptr(), y.data_ptr(), len(X), lr, want_loss=(s % every == 0))
            if loss is not None:
                hist.append(loss)
            if Xv is not None and (s + 1) % every == 0:
                vl = lbm.lbm_mlp_grad(m, xv.data_ptr(), yv.data_ptr(), len(Xv))
                if vl < best:
                    best, best_p = vl, lbm.lbm_mlp_get_params(m)
        p32, _ = best_p if best_p is not None else lbm.lbm_mlp_get_params(m)
    finally:
        lbm.lbm_mlp_destroy(m)
    p32 = fold_standardisation(p32, mX, sX, sY)
    return p32, p32.astype(np.float16), hist


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
    if body is not None:
        res["force_rms_fluctuation"], res["torque_rms_fluctuation"] = fluctuation(C[te], Fn[te], body[te], (cF, cM))
    print(json.dumps(res), flush=True)
    if args.out:
        np.savez(args.out, X=X, Y=Y, coarse=C, fine=Fn, params32=p32, params16=p16,
                 **({"body": body} if body is not None else {}))
    if args.params_out:
        np.save(args.params_out, p16)
    if args.eval_out:
        rec = {"force_rms": {k: res.get(f"force_rms_{k}") for k in ("without", "scaled", "with", "fluctuation", "fine")},
               "torque_rms": {k: res.get(f"torque_rms_{k}") for k in ("without", "scaled", "with", "fluctuation", "fine")},
               "units": "body-frame force in mu*gamma*a*b, torque in mu*gamma*a^2*b (RMS over held-out samples of the "
                        "vector error against the fine run)",
               "samples": {"total": res["samples"], "train": res["train"], "validation": res["validation"],
                           "held_out": res["held_out"]},
               "scale_factors": res["scale_factors"],
               "judge": "paired runs of the same prescribed body motion at minor semi-axis 6 lu (4x finer lattice, "
                        "16x the steps), window-averaged force and torque",
               "source": "python -m paper_1503_06869_gb300.closure_train " + " ".join(argv if argv is not None
                                                                                        else sys.argv[1:])}
        with open(args.eval_out, "w") as fh:
            json.dump(rec, fh, indent=1)
    return res


if __name__ == "__main__":
    main()

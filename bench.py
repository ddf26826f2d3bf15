#!/usr/bin/env python
"""Throughput of the fully resolved particle LBM time step on GB300.

One step = one pass of the whole hot path over the lattice: the fused D3Q19 TRT
stream-collide sweep with moving bounce-back and momentum exchange, the
rigid-body update and the obstacle re-mapping.  Default workload: the
256x128x128 shear cell (walls +-0.02, tau 0.8) with one spheroid a=24, b=3,
FP32 storage (offsets from the lattice weights).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the same workload instead (bounded sample).

Multi-GPU: one process per GPU (torchrun); each rank advances its own
independent replica of the workload (the single-lattice path has no data
exchange implemented), value = all ranks' cell updates / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from lbm_inputs import large_shear, small_shear, batched_shear, fibre_suspension, Particle  # noqa: E402

BYTES_PER_POP = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}

# DRAM traffic per sweep launch (dram__bytes_read.sum + dram__bytes_write.sum,
# mean of one even and one odd launch) from an ncu capture of the sweep
# kernel, keyed by workload and precision, with the fingerprint of the sweep
# sources it was taken on; a changed kernel reports no traffic until it is
# captured again.  Captures are summarised under profiles/.
SWEEP_SOURCES = ("paper_1503_06869_gb300/csrc/lbm_sweep.cuh", "paper_1503_06869_gb300/csrc/lbm_sweep.cu",
                 "paper_1503_06869_gb300/csrc/lbm_sweep_f32.cu", "paper_1503_06869_gb300/csrc/lbm_sweep_f16.cu",
                 "paper_1503_06869_gb300/csrc/lbm_sweep_bf16.cu", "paper_1503_06869_gb300/csrc/lbm_internal.cuh")
SWEEP_TRAFFIC = {
    ("shear256x128x128_spheroid24x3x3", "f32"): {"bytes": 569.97e6, "src": "3a1aa1b81564e284",
                                                "profile": "profiles/sweep_group_dram_shear256x128x128.md"},
    ("shear256x128x128_spheroid24x3x3", "f16"): {"bytes": 260.26e6, "src": "3a1aa1b81564e284",
                                                "profile": "profiles/sweep_group_dram_shear256x128x128.md"},
    ("shear256x128x128_spheroid24x3x3", "bf16"): {"bytes": 254.74e6, "src": "3a1aa1b81564e284",
                                                 "profile": "profiles/sweep_group_dram_shear256x128x128.md"},
    ("batched512_shear_cells", "f32"): {"bytes": 16697.4e6, "src": "3a1aa1b81564e284",
                                       "profile": "profiles/launches_batched512_f32.md"},
}


def sweep_fingerprint() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def sweep_traffic(workload_name: str, prec: str):
    rec = SWEEP_TRAFFIC.get((workload_name, prec))
    if rec is None or rec["src"] != sweep_fingerprint():
        return None
    return rec["bytes"]


def workload(name: str):
    if name == "large":
        return large_shear(seed=1)
    if name == "small":
        return small_shear(seed=1)
    if name == "batched":
        return batched_shear(seed=1)
    if name == "fibre":
        return fibre_suspension(seed=1)
    raise ValueError(name)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples (every 100 ms, time-stamped)
    kept only inside the windows marked with mark_start / mark_stop."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.windows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)  # the first sample precedes the timed region

    def mark_start(self):
        self.windows.append([time.time(), None])

    def mark_stop(self):
        if self.windows:
            self.windows[-1][1] = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        import datetime
        sm, mx, reasons, total = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            total += 1
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm_v = float(parts[2])
                mx = float(parts[3])
            except ValueError:
                continue
            if not any(w0 <= ts <= (w1 or ts) for w0, w1 in self.windows):
                continue
            sm.append(sm_v)
            for n, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": total,
                    "samples_in_timed_region": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": total, "samples_in_timed_region": len(sm)}


def dist_setup(n_gpus: int):
    """One process per GPU under torchrun: NCCL when CUDA is present, else
    gloo (host-side runs of the replica logic)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of N replicas (weak scaling): the units every rank
    processed, over the slowest rank's time, in millions per second."""
    return units_per_rank * world / (ms_max * 1e-3) / 1e6


def cpu_baseline(w, budget_s: float = 12.0, threads: int | None = None):
    """The oracle as it stands, timed on the host cores on a bounded sample of
    the workload: whole time steps of the first lattice, as many as fit in
    the time budget (at least one)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    lat = w.lattices[0]
    parts = [p for p in w.particles if p.cell == 0]
    for p in parts:
        p.cell = 0
    sim = oracle.Sim(lat, parts, openmp=True, threads=threads)
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter()
    per = t1 - t0
    n = max(0, int((budget_s - per) / max(per, 1e-9)))
    n = min(n, 200)
    if n:
        t0 = time.perf_counter()
        sim.step(n)
        t1 = time.perf_counter()
        per = (t1 - t0) / n
    steps = n if n else 1
    mlups = lat.ncells / per / 1e6
    return {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{steps} time step(s) of the {lat.nx}x{lat.ny}x{lat.nz} lattice "
                      f"with {len(parts)} particle(s), FP64 oracle, OpenMP over {threads} threads"}


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    budget = max(3.0, min(20.0, 2.0 * (args.steps + args.warmup)))
    cb = cpu_baseline(w, budget_s=budget)
    line = {"impl": "reference", "metric": "MLUPS", "value": cb["value"], "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, args, 0),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


L2_BYTES = 129e6  # GB300 L2


def l2_note(pop_bytes: float) -> str:
    """How the timed steps relate to L2: the populations are read and written
    once per step, so inputs larger than L2 need no flush between steps."""
    if pop_bytes > L2_BYTES:
        return "inputs larger than L2 (populations %.0f MB)" % (pop_bytes / 1e6)
    return "inputs fit in L2 (populations %.1f MB), not flushed: a parity-size case" % (pop_bytes / 1e6)


def config_of(w, args, nfluid):
    lat = w.lattices[0]
    cfg = {"workload": w.name, "lattices": len(w.lattices),
           "cells": int(w.ncells), "particles": len(w.particles), "precision": args.prec,
           "l2": l2_note(w.ncells * 19 * BYTES_PER_POP[args.prec]),
           "parallelism": f"replica x{args.gpus}",
           "closure": bool(getattr(args, "closure", False))}
    if len(w.lattices) == 1:
        cfg["lattice"] = [lat.nx, lat.ny, lat.nz]
        cfg["tau"] = lat.tau
    if nfluid:
        cfg["fluid_cells"] = int(nfluid)
    return cfg


def run_sequential(args, w, rank, world):
    """The lattices of a batch as independent contexts, each step launched
    lattice by lattice (the baseline the single batched launch replaces)."""
    import torch
    from paper_1503_06869_gb300 import lbm
    torch.cuda.set_device(0)
    sims = []
    for c, lat in enumerate(w.lattices):
        parts = [Particle(**{**p.__dict__, "cell": 0}) for p in w.particles if p.cell == c]
        sims.append(lbm.Simulation([lat], parts, prec=args.prec))
    for _ in range(args.warmup):
        for s in sims:
            s.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in sims:
            s.step(1)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    value = w.ncells * args.steps / el / 1e6
    line = {"metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el * 1e3 / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {**config_of(w, args, 0), "mode": "sequential single-lattice contexts"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s in sims:
        s.close()
    return 0


PREC_NAMES = {"f64": "f64", "f32": "f32", "f16": "f16", "bf16": "bf16"}


def fluid_cells(lbm, h, lattices):
    n = 0
    for c, lat in enumerate(lattices):
        f = lbm.lbm_get_fields(h, lat.ncells, c, rho=False, u=False, flags=True, pid=False)
        n += int((f["flags"] == 0).sum())
    return n


def timed_steps(sim, lbm, steps, world, clocks, min_region_s, max_reps=400):
    """Repeat the timed region -- exactly `steps` steps (CUDA-graph replay),
    bracketed by a barrier and a device synchronisation on both sides, CUDA
    events on the context's stream -- until the repetitions cover about
    min_region_s; returns the per-repetition times (ms, max over ranks) and
    the kernels launched per repetition."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times, launches = [], 0
    total = 0.0
    while True:
        l0 = lbm.lbm_get_launch_count(sim.h)
        barrier(world)
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.mark_start()
        ev0.record(sim.stream)
        sim.step(steps)
        ev1.record(sim.stream)
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.mark_stop()
        barrier(world)
        launches = lbm.lbm_get_launch_count(sim.h) - l0
        ms = max_over_ranks(ev0.elapsed_time(ev1), world)
        times.append(ms)
        total += ms
        # every rank takes the same decision (the times are the max over ranks)
        if total >= 1e3 * min_region_s or len(times) >= max_reps:
            break
    return times, launches


def measure(args, w, prec, world, local, launch=None, cpt=None, closure_params=None, clocks=None,
            min_region_s=1.0, steps=None, e2e_steps=0):
    """One workload in one storage form: autotuned launch, warm-up, the timed
    repetitions, the sweep kernel timed alone (eager launches with CUDA events
    around every sweep), optionally the end-to-end loop through the C
    interface with host buffers.  Returns a dict of results."""
    import torch
    from paper_1503_06869_gb300 import lbm
    steps = steps or args.steps
    sim = lbm.Simulation(w.lattices, w.particles, prec=prec, device=local)
    h = sim.h
    if closure_params is not None:
        lbm.lbm_set_closure(h, closure_params)
    if args.remap_fused:
        lbm.lbm_set_remap_fused(h, True)
    if launch is None:
        lbm.lbm_autotune(h)
    else:
        lbm.lbm_set_launch(h, launch, 0)
        if cpt:
            lbm.lbm_set_cells_per_thread(h, cpt)
        if getattr(args, "split", False):
            lbm.lbm_set_sweep_split(h, True)
        lbm.lbm_set_sweep_prefetch(h, ["off", "all", "even", "odd"].index(getattr(args, "prefetch", "off")))
    info = lbm.lbm_get_info(h)
    sim.step(args.warmup)
    sim.sync()
    nfluid = fluid_cells(lbm, h, w.lattices)
    times, launches = timed_steps(sim, lbm, steps, world, clocks, min_region_s)
    ms_rep = statistics.median(times)
    ms_step = ms_rep / steps

    # the sweep kernel alone: the same number of steps again, every sweep
    # launch bracketed by CUDA events on the context's stream (eager launches:
    # a graph replay has no events between its kernels)
    lbm.lbm_set_sweep_timing(h, True)
    sim.step(steps)
    sweep_ms, sweep_n = lbm.lbm_get_sweep_timing(h)
    lbm.lbm_set_sweep_timing(h, False)
    sim.sync()

    peak, peak_kind = measured_peaks()
    bpp = BYTES_PER_POP[prec]
    bytes_per_launch = 38 * bpp * nfluid
    sweep_avg_ms = sweep_ms / max(sweep_n, 1)
    achieved = bytes_per_launch / (sweep_avg_ms * 1e-3) / 1e9
    step_achieved = bytes_per_launch / (ms_step * 1e-3) / 1e9
    res = {"workload": w.name, "prec": prec, "cells": int(w.ncells), "fluid_cells": int(nfluid),
           "particles": len(w.particles), "ms_per_step": ms_step, "reps": len(times), "steps_per_rep": steps,
           "rep_ms_min": min(times), "rep_ms_max": max(times), "launches_per_rep": int(launches),
           "mlups": w.ncells * steps * world / (ms_rep * 1e-3) / 1e6,
           "fluid_mlups": nfluid * steps * world / (ms_rep * 1e-3) / 1e6,
           "particle_steps_per_s": len(w.particles) * steps * world / (ms_rep * 1e-3),
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "traffic": sweep_traffic(w.name, prec),
                        "kernel": "sweep", "bytes_per_launch": bytes_per_launch,
                        "avg_launch_ms": round(sweep_avg_ms, 5),
                        "avg_launch_source": "eager pass of the same step count, CUDA events around every "
                                             "sweep launch on the context's stream",
                        "step_achieved": round(step_achieved, 1), "step_frac": round(step_achieved / peak, 4),
                        "peak_kind": f"{peak_kind} hbm_gbs"},
           "launch": {"block": info.sweep_block, "grid": info.sweep_grid, "cells_per_thread": info.cells_per_thread,
                      "split": bool(info.sweep_split), "remap_fused": bool(info.remap_fused),
                      "l2_prefetch": ["off", "all", "even steps", "odd steps"][info.sweep_prefetch_mode]}}
    if e2e_steps:
        # every step: H2D of the particles' external loads from pinned memory,
        # the step, D2H of the hydrodynamic force/torque (synchronising)
        npart = max(len(w.particles), 1)
        ext = torch.zeros((npart, 3), dtype=torch.float64).pin_memory()
        Fh = torch.zeros((npart, 3), dtype=torch.float64).pin_memory()
        Mh = torch.zeros((npart, 3), dtype=torch.float64).pin_memory()
        extn, Fn, Mn = ext.numpy(), Fh.numpy(), Mh.numpy()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            lbm.lbm_set_external(h, extn, None, len(w.particles))
            lbm.lbm_step(h, 1)
            lbm.lbm_get_forces(h, len(w.particles), Fn, Mn)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2e_s = max_over_ranks(t1 - t0, world)
        res["e2e"] = {"value": round(w.ncells * e2e_steps * world / e2e_s / 1e6, 1), "unit": "MLUPS",
                      "h2d_bytes_per_step": 24 * len(w.particles), "d2h_bytes_per_step": 48 * len(w.particles),
                      "steps": e2e_steps}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return res


def secondary(args, world, local):
    """The other workloads of the benchmark on the same GPU, each in its own
    timed region: FP16 and BF16 offset storage of the 256x128x128 cell, the
    512-lattice batch (FP32) and the 2,000-spheroid fibre suspension (FP32,
    learned closure on with the trained parameters when they are present)."""
    out = {}
    w = workload("large")
    for prec in ("f16", "bf16"):
        r = measure(args, w, prec, world, local, min_region_s=0.5, steps=max(args.steps, 20))
        out[f"storage_{prec}"] = summarise(r)
    wb = workload("batched")
    r = measure(args, wb, "f32", world, local, min_region_s=0.5, steps=max(args.steps // 4, 4))
    out["batched"] = summarise(r)
    wf = workload("fibre")
    params = trained_closure()
    r = measure(args, wf, "f32", world, local, closure_params=params, min_region_s=0.5,
                steps=max(args.steps // 4, 4))
    s = summarise(r)
    s["closure"] = "trained" if params is not None else "off"
    err = closure_error_record()
    if err is not None:
        s["force_torque_error"] = err
    out["fibre"] = s
    return out


def summarise(r):
    keep = ("workload", "prec", "cells", "fluid_cells", "particles", "ms_per_step", "reps", "steps_per_rep",
            "mlups", "particle_steps_per_s", "launch")
    s = {k: r[k] for k in keep}
    s["mlups"] = round(s["mlups"], 1)
    s["particle_steps_per_s"] = round(s["particle_steps_per_s"], 1)
    s["ms_per_step"] = round(s["ms_per_step"], 5)
    rf = r["roofline"]
    s["roofline"] = {k: rf[k] for k in ("achieved", "peak", "frac", "avg_launch_ms", "bytes_per_launch",
                                        "step_frac", "traffic")}
    return s


CLOSURE_PARAMS_FILE = os.path.join(ROOT, "paper_1503_06869_gb300", "closure", "params_fp16.npy")
CLOSURE_EVAL_FILE = os.path.join(ROOT, "paper_1503_06869_gb300", "closure", "evaluation.json")


def trained_closure():
    if os.path.exists(CLOSURE_PARAMS_FILE):
        return np.load(CLOSURE_PARAMS_FILE).astype(np.float16)
    return None


def closure_error_record():
    """Held-out force/torque error of the coarse runs against the fine judge,
    with and without the trained closure, as the training driver wrote it."""
    if not os.path.exists(CLOSURE_EVAL_FILE):
        return None
    d = json.load(open(CLOSURE_EVAL_FILE))
    return {k: d[k] for k in d if k in ("force_rms", "torque_rms", "units", "samples", "judge", "source")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "small", "batched", "fibre"])
    ap.add_argument("--sequential", action="store_true",
                    help="batched workload: one context per lattice, stepped one after another")
    ap.add_argument("--closure", action="store_true",
                    help="enable the learned force/torque closure (trained parameters when present, else "
                         "seeded small ones)")
    ap.add_argument("--prec", default="f32", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--min-region-s", type=float, default=1.0,
                    help="repeat the K-step timed region until the repetitions cover this many seconds")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the FP16/BF16, batched and fibre-suspension lines of the default run")
    ap.add_argument("--launch", type=int, default=None,
                    help="fixed sweep block size (0 ring, -1 staged, 32..256 direct) instead of the autotuner's "
                         "choice; for profiling runs, where the profiler's serialisation skews the autotuner")
    ap.add_argument("--cpt", type=int, default=None, help="with --launch: cells per thread of the direct sweep")
    ap.add_argument("--split", action="store_true",
                    help="with --launch: near-obstacle cells in a kernel of their own (split sweep)")
    ap.add_argument("--prefetch", default="off", choices=["off", "all", "even", "odd"],
                    help="with --launch: L2 prefetch of a later tile in every sweep, or in the even- or odd-step "
                         "sweeps only")
    ap.add_argument("--remap-fused", action="store_true",
                    help="run the re-mapping step as one cooperative launch instead of five launches")
    args = ap.parse_args()
    rank, world, local = dist_setup(args.gpus)
    w = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    if args.sequential:
        return run_sequential(args, w, rank, world)

    import torch
    torch.cuda.set_device(local)
    params = None
    if args.closure:
        params = trained_closure()
        if params is None:
            # throughput only: seeded small parameters
            from paper_1503_06869_gb300 import lbm
            params = (np.random.default_rng(0).normal(size=lbm.CLOSURE_PARAMS) * 0.01).astype(np.float16)
    clocks = ClockSampler(local)
    clocks.start()
    r = measure(args, w, args.prec, world, local, launch=args.launch, cpt=args.cpt, closure_params=params,
                clocks=clocks, min_region_s=args.min_region_s, e2e_steps=args.e2e_steps)
    clk = clocks.stop()
    line = {"metric": "MLUPS", "value": round(r["mlups"], 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(r["ms_per_step"], 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic", "config": config_of(w, args, r["fluid_cells"]),
            "timing": {"reps": r["reps"], "steps_per_rep": r["steps_per_rep"], "statistic": "median rep",
                       "rep_ms_min": round(r["rep_ms_min"], 4), "rep_ms_max": round(r["rep_ms_max"], 4)},
            "fluid_mlups": round(r["fluid_mlups"], 1),
            "particle_steps_per_s": round(r["particle_steps_per_s"], 1),
            "roofline": r["roofline"],
            "e2e": r["e2e"],
            "gpu_launches": r["launches_per_rep"],
            "launch": r["launch"],
            "clocks": clk}
    if world == 1 and not args.no_secondary and args.workload == "large" and args.launch is None:
        line["secondary"] = secondary(args, world, local)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

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
SWEEP_SOURCES = ("paper_1503_06869_gb300/csrc/lbm_sweep.cu", "paper_1503_06869_gb300/csrc/lbm_internal.cuh")
SWEEP_TRAFFIC = {
    ("shear256x128x128_spheroid24x3x3", "f32"): {"bytes": 570.72e6, "src": "3e5fec48d2252c95",
                                                "profile": "profiles/sweep_kernel_shear256x128x128_f32.md"},
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
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "small", "batched", "fibre"])
    ap.add_argument("--sequential", action="store_true",
                    help="batched workload: one context per lattice, stepped one after another")
    ap.add_argument("--closure", action="store_true",
                    help="enable the learned force/torque closure (seeded small parameters)")
    ap.add_argument("--prec", default="f32", choices=["f64", "f32", "f16", "bf16"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch", type=int, default=None,
                    help="fixed sweep block size (0 ring, -1 staged, 32..256 direct) instead of the autotuner's "
                         "choice; for profiling runs, where the profiler's serialisation skews the autotuner")
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
    from paper_1503_06869_gb300 import lbm
    torch.cuda.set_device(local)
    sim = lbm.Simulation(w.lattices, w.particles, prec=args.prec, device=local)
    h = sim.h
    if args.closure:
        # throughput only: the parameters are seeded and small, not trained
        theta = np.random.default_rng(0).normal(size=lbm.CLOSURE_PARAMS) * 0.01
        lbm.lbm_set_closure(h, theta.astype(np.float16))
    if args.remap_fused:
        lbm.lbm_set_remap_fused(h, True)
    if args.launch is None:
        lbm.lbm_autotune(h)
    else:
        lbm.lbm_set_launch(h, args.launch, 0)
    info = lbm.lbm_get_info(h)
    sim.step(args.warmup)
    sim.sync()
    nfluid = 0
    for c, lat in enumerate(w.lattices[:1]):
        f = lbm.lbm_get_fields(h, lat.ncells, c, rho=False, u=False, flags=True, pid=False)
        nfluid = int((f["flags"] == 0).sum())
    fluid_total = nfluid if len(w.lattices) == 1 else None

    # --- timed region: K whole steps (CUDA-graph replay), inputs resident in
    # HBM and larger than L2 -------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches0 = lbm.lbm_get_launch_count(h)
    barrier(world)
    torch.cuda.synchronize()
    ev0.record(sim.stream)
    sim.step(args.steps)
    ev1.record(sim.stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = lbm.lbm_get_launch_count(h) - launches0

    # --- the sweep kernel alone: the same K steps again, each sweep launch
    # bracketed by CUDA events on the context's stream (eager launches) -----
    lbm.lbm_set_sweep_timing(h, True)
    sim.step(args.steps)
    sweep_ms, sweep_n = lbm.lbm_get_sweep_timing(h)
    lbm.lbm_set_sweep_timing(h, False)
    ms_max = max_over_ranks(ms, world)
    cells = w.ncells
    value = whole_job_rate(cells * args.steps, world, ms_max)

    # roofline of the sweep kernel (dominant kernel): algorithmic bytes =
    # 19 loads + 19 stores per fluid cell update
    peak, peak_kind = measured_peaks()
    bpp = BYTES_PER_POP[args.prec]
    if fluid_total is None:
        fluid_total = 0
        for c, lat in enumerate(w.lattices):
            f = lbm.lbm_get_fields(h, lat.ncells, c, rho=False, u=False, flags=True, pid=False)
            fluid_total += int((f["flags"] == 0).sum())
    bytes_per_launch = 38 * bpp * fluid_total
    sweep_avg_ms = sweep_ms / max(sweep_n, 1)
    achieved = bytes_per_launch / (sweep_avg_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": sweep_traffic(w.name, args.prec),
            "kernel": "sweep_kernel", "bytes_per_launch": bytes_per_launch,
            "avg_launch_ms": round(sweep_avg_ms, 5), "peak_kind": f"{peak_kind} hbm_gbs"}

    # --- end-to-end through the C interface with host buffers -------------
    # every step: H2D of the particles' external loads from pinned memory,
    # the step, D2H of the hydrodynamic force/torque (synchronising)
    npart = max(len(w.particles), 1)
    ext = torch.zeros((npart, 3), dtype=torch.float64).pin_memory()
    Fh = torch.zeros((npart, 3), dtype=torch.float64).pin_memory()
    Mh = torch.zeros((npart, 3), dtype=torch.float64).pin_memory()
    extn, Fn, Mn = ext.numpy(), Fh.numpy(), Mh.numpy()
    e2e_steps = args.e2e_steps
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
    e2e_val = cells * e2e_steps * world / e2e_s / 1e6

    line = {"metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic", "config": config_of(w, args, fluid_total),
            "fluid_mlups": round(fluid_total * args.steps * world / (ms_max * 1e-3) / 1e6, 1),
            "particle_steps_per_s": round(len(w.particles) * args.steps * world / (ms_max * 1e-3), 1),
            "roofline": roof,
            "e2e": {"value": round(e2e_val, 1), "unit": "MLUPS",
                    "h2d_bytes_per_step": 24 * len(w.particles),
                    "d2h_bytes_per_step": 48 * len(w.particles)},
            "gpu_launches": int(launches),
            "launch": {"block": info.sweep_block, "grid": info.sweep_grid, "split": bool(info.sweep_split),
                       "remap_fused": bool(info.remap_fused), "remap_grid": info.remap_grid},
            "clocks": clk}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

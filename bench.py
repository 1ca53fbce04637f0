#!/usr/bin/env python3
"""Benchmark of the homogenized LB rotor time step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

A step is one pass of the whole hot path (listing "HHRRLBM-FSI"): porosity
embedding + wall model of the rotor box, fused collide-and-stream of every
cell, momentum-exchange force/torque reduction, and the FP64 mass check
every 100 steps.  Workload: the 256x256x512 D3Q19 rotor (FP32 populations,
single-buffer AA pattern, R = 64 NACA 4412 three-bladed rotor at TSR 6,
5 % synthetic turbulent inflow).  Prints one JSON line (rank 0).

Under torchrun (N > 1) the lattice is decomposed along the flow axis (the
paper's weak scaling, one rotor per GPU): a row of N rotor256 domains,
256x256x(512 N) cells with a rotor every 512 planes, one slab of 512 planes
per rank; every odd step exchanges the halo planes between neighbouring
ranks (NCCL point-to-point) and the per-rotor loads are reduced.  The timed
region is bracketed by barriers and the max over ranks is reported.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline (FP32 vs 16-bit store); adjoint/forward step ratio"
UNIT = "MLUPS"
WORKLOAD_DESC = ("rotor256: 256x256x512 cells (33.5M), D3Q19, FP32 weight-shifted populations, "
                 "AA single buffer, one 3-blade NACA4412 rotor R=64 at TSR 6, 5% turbulent inflow "
                 "(64 Fourier modes), tau_mo 0.5005, C_S 0.1, Spalding wall model")


# --------------------------------------------------------------------------
# distributed helpers (barrier + max over ranks)
# --------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(backend: str):
    import torch.distributed as dist
    world, rank, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return world, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([float(x)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return float(x)


def aggregate(elapsed_s: float, cells: int, steps: int, world: int, device="cpu"):
    """Whole-job throughput: all ranks' cell updates over the slowest rank's time."""
    t = max_over_ranks(elapsed_s, device)
    return world * cells * steps / t / 1e6, t


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on a bounded sample
# --------------------------------------------------------------------------
def oracle_sample(steps: int, crop=(160, 160, 72), warmup: int = 1):
    """Time the oracle on a crop of the rotor256 workload centred on the rotor
    (same rotor, inflow table and parameters; the crop's lateral faces are
    periodic).  Returns (MLUPS, seconds, threads, description)."""
    cores = len(os.sched_getaffinity(0))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle as O
    import workloads as W
    wl = W.workload("rotor256")
    nx, ny, nz = crop
    spec = wl.rotors[0]
    grid = wl.blade_grids()[0]
    center = (0.5 * (nx - 1), 0.5 * (ny - 1), 0.5 * nz)
    rot = O.make_rotor(grid, center=center, axis=2, omega=spec.omega(wl.u_in), phase0=spec.phase0)
    o = O.Oracle(nx, ny, nz, tau_mo=wl.tau_mo, c_smag=wl.c_smag, u_in=wl.u_in, eps_h=wl.eps_h,
                 modes=wl.modes(), rotors=[rot])
    o.step(max(1, warmup))         # includes the first touch of the FP64 arrays
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    cells = nx * ny * nz
    whole = min(nx, ny) > 2 * (spec.radius + 4)
    what = "the whole rotor" if whole else "the hub and inner blade span"
    threads = int(os.environ["OMP_NUM_THREADS"])
    desc = (f"FP64 oracle, {steps} steps (after {max(1, warmup)} warm-up) of a {nx}x{ny}x{nz} crop of "
            f"rotor256 containing {what} (same rotor, inflow modes and parameters), {threads} OpenMP threads")
    return cells * steps / dt / 1e6, dt, threads, desc


def run_reference(args):
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    steps = max(1, args.steps)
    # each step is one oracle step on the crop; the crop shrinks for long runs
    crop = (160, 160, 72) if steps <= 200 else (96, 96, 48)
    mlups, dt, cores, desc = oracle_sample(steps, crop, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * dt / steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "sample": desc},
        "cpu_baseline": {"value": round(mlups, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(mlups, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# CUDA arm
# --------------------------------------------------------------------------
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one bulk collide
# launch of the rotor256 step from one ncu capture (the mean of an even- and
# an odd-step launch where both were captured), per (storage, layout);
# reported only while the kernel sources hash to the value they had at the
# capture (else null)
NCU_TRAFFIC = {"source_sha": "152c587229e90350",
               "bytes_per_launch": {("f32", "aa"): 4872067840, ("f16s", "aa_halves"): 2484081792}}


def inflow_planes_pinned(wl, t0, n, dev):
    """The workload's synthetic inflow on the inlet plane for steps t0 .. t0+n-1
    (U a + sum_m a_m cos(k.x') + b_m sin(k.x'), x' = x - U t a), shaped
    (n, 3, n_c, n_b) as Lattice.inflow_plane_shape(), in pinned host memory:
    the per-step input of the end-to-end run.  Evaluated on the device in
    FP64 to keep the preparation short; it is input data, outside any timed
    region."""
    import torch
    a = wl.flow_axis
    b, c = (a + 1) % 3, (a + 2) % 3
    shape = wl.shape
    nb, nc = shape[b], shape[c]
    modes = wl.modes()
    out = torch.empty((n, 3, nc, nb), dtype=torch.float32).pin_memory()
    X = torch.zeros((3, nc, nb), dtype=torch.float64, device=dev)
    X[b] = torch.arange(nb, dtype=torch.float64, device=dev)[None, :]
    X[c] = torch.arange(nc, dtype=torch.float64, device=dev)[:, None]
    md = None if modes is None else torch.as_tensor(modes, dtype=torch.float64, device=dev)
    for i in range(n):
        X[a] = -wl.u_in * (t0 + i)
        u = torch.zeros((3, nc, nb), dtype=torch.float64, device=dev)
        u[a] = wl.u_in
        if md is not None:
            ph = torch.einsum("mk,kcb->mcb", md[:, 0:3], X)
            u += torch.einsum("mk,mcb->kcb", md[:, 3:6], torch.cos(ph)) + \
                torch.einsum("mk,mcb->kcb", md[:, 6:9], torch.sin(ph))
        out[i].copy_(u.float())
    return out


def bulk_kernel_name(wl, layout="aa") -> str:
    """The kernel of the bulk collide-and-stream launch: cell pairs in packed
    FP32x2 arithmetic when nx is even (x-adjacent pairs; (x, x + nx/2) in the
    AA layout with x halves), one cell per thread otherwise."""
    if wl.nx % 2:
        return "collide_kernel"
    return "collide_halves_kernel" if layout == "aa_halves" else "collide_pair_kernel"


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("hl_device.cuh", "hl_pair.cuh", "hl_kernels.cu", "hl_internal.h"):
        with open(os.path.join(ROOT, "paper_2510_13726_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def chain_workload(base, n):
    """A row of n copies of a workload along its flow axis z (rotor k at the
    base rotor's position plus k lengths): the weak-scaling lattice."""
    import dataclasses
    from workloads.configs import RotorSpec
    rot = [dataclasses.replace(r, center=(r.center[0], r.center[1], r.center[2] + k * base.nz))
           for k in range(n) for r in base.rotors]
    return dataclasses.replace(base, nz=base.nz * n, rotors=rot, name=f"{base.name}_row{n}",
                               note=f"{n} x {base.name} along the flow axis, one slab per rank")


def run_cuda_slabs(args, world, rank, local, dev):
    """N > 1: one slab of the rotor row per rank, halo exchange every odd step."""
    import torch
    import torch.distributed as dist
    import workloads as W
    from paper_2510_13726_b300.slabs import SlabDomain

    base = W.workload(args.workload)
    if base.flow_axis != 2:
        raise SystemExit("the multi-GPU run decomposes along z: choose a workload that flows along z")
    wl = chain_workload(base, world)
    cuts = [k * base.nz for k in range(world + 1)]
    dom = SlabDomain.from_workload(wl, cuts=cuts, held=[rank], rank_of=list(range(world)),
                                   group=dist.group.WORLD, storage=args.storage, device=dev)
    lat = dom.engines[rank]
    K, Wm = args.steps, args.warmup
    dom.step(Wm)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lat.profile_begin(4 * K + 16)
    e0.record(lat.stream)
    dom.step(K)
    e1.record(lat.stream)
    e1.synchronize()
    prof = lat.profile_end()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    cells_rank = wl.nx * wl.ny * (cuts[rank + 1] - cuts[rank])
    value, t_max = aggregate(elapsed, cells_rank, K, world, device=dev)
    # end to end: every step the inlet slab takes the step's inflow plane from
    # pinned host memory, and every rank reads the reduced loads of every rotor
    K2 = max(1, min(K, 200))
    plane = None
    if rank == 0:
        host_planes = inflow_planes_pinned(base, lat.t, K2, dev)
        plane = torch.empty(lat.inflow_plane_shape(), dtype=torch.float32, device=dev)
        lat.set_inflow_plane(plane)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for i in range(K2):
        if plane is not None:
            with torch.cuda.stream(lat.stream):
                plane.copy_(host_planes[i], non_blocking=True)
        dom.step(1)
        F, Fa, M, Ma = dom.loads()
    t_e2e = time.perf_counter() - t0
    e2e_value, _ = aggregate(t_e2e, cells_rank, K2, world, device=dev)
    launches = sum(n for _, n in prof.values())
    kernels = {k: {"launches": n, "ms_per_launch": round(ms / n, 4) if n else None} for k, (ms, n) in prof.items()}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": round(1e3 * t_max / K, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage == "f32" else "f32-math/" + args.storage, "data": "synthetic",
            "config": {"workload": f"{world} x rotor256 along the flow axis: 256x256x{wl.nz} cells, "
                                   f"{world} rotors 512 planes apart (one per rank); " + WORKLOAD_DESC,
                       "name": wl.name, "cells": wl.cells, "cells_per_rank": cells_rank, "q": wl.q,
                       "storage": args.storage, "layout": "aa",
                       "parallelism": f"slabs x{world} along z (halo exchange every odd step, NCCL p2p)",
                       "l2": "no flush: the populations exceed the 126 MB L2"},
            "kernels_rank0": kernels, "gpu_launches": launches, "clocks": clk,
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                    "h2d_bytes_per_step": plane.numel() * 4, "d2h_bytes_per_step": 12 * 8 * len(wl.rotors) * world,
                    "steps": K2, "per_step": "inflow plane to the inlet slab from pinned host memory, one step "
                                             "of every slab with its halo exchange, the reduced loads of every "
                                             "rotor to the host on every rank"},
            "thrust": [float(v) for v in F[:, 2]],
            "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    dom.close()
    return 0


def run_cuda(args):
    import torch
    import workloads as W
    from paper_2510_13726_b300 import Lattice
    from paper_2510_13726_b300.perf import collide_bytes

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_init("nccl")
    dev = torch.device("cuda", local)
    if world > 1:
        return run_cuda_slabs(args, world, rank, local, dev)

    wl = W.workload(args.workload)
    lat = Lattice.from_workload(wl, storage=args.storage, layout=args.layout, device=dev)
    stream = lat.stream
    K, Wm = args.steps, args.warmup
    lat.step(Wm)

    # ---- device-timed region ------------------------------------------------
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lat.profile_begin(4 * K + 16)
    e0.record(stream)
    lat.step_async(K)
    e1.record(stream)
    e1.synchronize()
    prof = lat.profile_end()
    lat.check()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    barrier()
    elapsed = e0.elapsed_time(e1) / 1e3
    value, t_max = aggregate(elapsed, wl.cells, K, world, device=dev)

    # ---- roofline of the dominant kernel (collide-and-stream) ----------------
    box_cells = wall_cells = 0
    for k in range(lat.nrot):
        band = lat.rotor_band(k)
        box_cells += int(band["d"].numel())
        wall_cells += int(((band["flags"] & 2) > 0).sum().item())
    if prof["collide_box"][1] > 0:
        # overlap on: the timed collide launch covers the cells outside every rotor box
        alg_bytes = collide_bytes(wl.q, args.storage, wl.cells - box_cells)
        roof_cells = wl.cells - box_cells
    else:
        alg_bytes = collide_bytes(wl.q, args.storage, wl.cells, box_cells, wall_cells)
        roof_cells = wl.cells
    # algorithmic bytes of all collide-and-stream work of one step (every cell)
    step_bytes = collide_bytes(wl.q, args.storage, wl.cells, box_cells, wall_cells)
    c_ms, c_n = prof["collide"]
    per_launch_s = c_ms / c_n / 1e3
    achieved = alg_bytes / per_launch_s / 1e9
    peak, peak_src = measured_peaks()
    sha = kernel_source_sha()
    traffic = (NCU_TRAFFIC["bytes_per_launch"].get((args.storage, args.layout))
               if NCU_TRAFFIC["source_sha"] == sha and args.workload == "rotor256" else None)
    total_kernel_ms = sum(v[0] for v in prof.values())
    kernels = {k: {"launches": n, "ms_per_launch": round(ms / n, 4) if n else None,
                   "share": round(ms / total_kernel_ms, 4) if total_kernel_ms else None}
               for k, (ms, n) in prof.items()}
    launches = sum(n for _, n in prof.values())

    # ---- end to end through the public API with host buffers ----------------
    # per step: hl_step (launches + stream sync + device error word to host)
    # and hl_forces / hl_moments into host arrays (thrust and torque every step)
    # pipelined: every step, the inflow plane of that step copied from pinned
    # host memory into the lattice's caller-supplied inflow buffer, the step
    # enqueued (hl_step_async), and its thrust and torque copied back into a
    # two-slot pinned ring that the host reads two steps later; the device
    # error word is checked once at the end (hl_check)
    K2 = max(1, min(K, 200))
    inflow = bool(lat.cfg.open_boundaries)
    if inflow:
        host_planes = inflow_planes_pinned(wl, lat.t, K2, dev)
        plane = torch.empty(lat.inflow_plane_shape(), dtype=torch.float32, device=dev)
        lat.set_inflow_plane(plane)
    nr = max(1, lat.nrot)
    ring = torch.zeros((2, nr, 6), dtype=torch.float64).pin_memory()
    done = [torch.cuda.Event(), torch.cuda.Event()]
    loads = np.zeros((K2, nr, 6))
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for i in range(K2):
        slot = i & 1
        if inflow:
            with torch.cuda.stream(lat.stream):
                plane.copy_(host_planes[i], non_blocking=True)
        lat.step_async(1)
        if i >= 2:
            done[slot].synchronize()
            loads[i - 2] = ring[slot].numpy()
        lat.loads_async(ring[slot])
        done[slot].record(lat.stream)
    lat.check()
    for i in range(max(0, K2 - 2), K2):
        loads[i] = ring[i & 1].numpy()
    t_e2e = time.perf_counter() - t0
    if inflow:
        lat.set_inflow_plane(None)
    F, Fa = lat.forces()
    assert np.array_equal(loads[-1, :lat.nrot, 0:3], F), "pipelined loads disagree with hl_forces"
    e2e_value, _ = aggregate(t_e2e, wl.cells, K2, world, device=dev)
    h2d = plane.numel() * 4 if inflow else 0    # the step's inflow plane
    d2h = 6 * 8 * lat.nrot                       # each step's F and M per rotor (the error word once per run)

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            mlups, dt, cores, desc = oracle_sample(args.cpu_steps)
            cpu = {"value": round(mlups, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": round(1e3 * t_max / K, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else "f32-math/" + args.storage,
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC if args.workload == "rotor256" else wl.note,
                       "name": args.workload, "cells": wl.cells, "q": wl.q, "storage": args.storage, "layout": args.layout,
                       "rotors": len(wl.rotors), "parallelism": "single GPU",
                       "l2": "no flush: the populations (%.2f GB) exceed the 126 MB L2" %
                             (wl.cells * wl.q * (4 if args.storage == "f32" else 2) / 1e9)},
            "roofline": {"bound": "hbm", "kernel": bulk_kernel_name(wl, args.layout), "achieved": round(achieved, 1),
                         "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                         else "fallback", "traffic": traffic,
                         "alg_bytes_per_launch": alg_bytes, "cells_per_launch": roof_cells,
                         "step_effective_gbs": round(step_bytes / (t_max / K) / 1e9, 1),
                         "step_effective_frac": round(step_bytes / (t_max / K) / 1e9 / peak, 4),
                         "frac_of_8TBps_nominal": round(achieved / 8000.0, 4)},
            "kernels": kernels,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": K2,
                    "per_step": "inflow plane from pinned host memory (hl_set_inflow_plane buffer), "
                                "hl_step_async, the step's F and M per rotor to pinned host memory "
                                "(hl_loads_async, read by the host two steps later); hl_check (error "
                                "word) at the end"},
            "thrust_last": float(F[0, wl.flow_axis]) if lat.nrot else None,
            "cpu_baseline": cpu,
        }
        extras = set() if args.no_extra else set(args.extras.split(","))
        if world == 1 and extras:
            lat.close()
            torch.cuda.empty_cache()
            if "storage" in extras:
                line["storage_study"] = storage_study(dev, args.extra_steps)
            if "farm" in extras:
                line["farm"] = farm_run(dev, args.extra_steps)
            if "adjoint" in extras and args.adjoint_steps > 0:
                S = args.adjoint_steps
                line["adjoint"] = adjoint_run(dev, S, max(1, S // 4), min(100, max(2, S // 2)))
            if "driven" in extras:
                line["driven_rotor"] = driven_run(dev, 200)
            if args.farm_wake_steps > 0:
                line["farm_wake"] = farm_wake(dev, args.farm_wake_steps)
        print(json.dumps(line), flush=True)
    lat.close()
    return 0


def timed_run(wl, storage, steps, warmup, dev, layout="aa"):
    """MLUPS of `steps` steps of a workload (CUDA events on the lattice stream)
    and the per-launch roofline of its collide-and-stream launch."""
    import torch
    from paper_2510_13726_b300 import Lattice
    from paper_2510_13726_b300.perf import collide_bytes
    lat = Lattice.from_workload(wl, storage=storage, layout=layout, device=dev)
    lat.step(warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    lat.profile_begin(4 * steps + 16)
    e0.record(lat.stream)
    lat.step_async(steps)
    e1.record(lat.stream)
    e1.synchronize()
    prof = lat.profile_end()
    lat.check()
    ms = e0.elapsed_time(e1) / steps
    box = sum(lat.rotor_box(k)[1][0] * lat.rotor_box(k)[1][1] * lat.rotor_box(k)[1][2] for k in range(lat.nrot))
    cells = wl.cells - box if prof["collide_box"][1] else wl.cells
    c_ms, c_n = prof["collide"]
    peak, _ = measured_peaks()
    gbs = collide_bytes(wl.q, storage, cells) / (c_ms / c_n / 1e3) / 1e9
    F, _ = lat.forces()
    M, _ = lat.moments()
    lat.close()
    del lat
    torch.cuda.empty_cache()
    return {"layout": layout, "MLUPS": round(wl.cells / ms / 1e3, 1), "ms_per_step": round(ms, 4),
            "collide_gbs": round(gbs, 1), "collide_frac": round(gbs / peak, 4),
            "thrust_last": [round(float(f[wl.flow_axis]), 6) for f in F],
            "torque_last": [round(float(m[wl.flow_axis]), 6) for m in M]}


def storage_study(dev, steps):
    """FP32 vs FP16 / BF16 storage: the D3Q27 512x512x1024 rotor (R = 128,
    TSR 7) and the D3Q19 256x256x512 benchmark rotor (R = 64, TSR 6, 5 %
    turbulence; at least 200 steps).  Each storage form in its faster
    layout: FP32 in the AA layout, 16-bit storage in the AA layout with x
    halves (every bulk access aligned; the plain AA layout is reported
    beside it)."""
    import workloads as W

    def study(wl, desc, n, warm):
        out = {"workload": desc, "steps": n, "f32": timed_run(wl, "f32", n, warm, dev)}
        for st in ("f16s", "bf16s"):
            out[st] = timed_run(wl, st, n, warm, dev, layout="aa_halves")
            out[f"ratio_{st}_over_f32"] = round(out[st]["MLUPS"] / out["f32"]["MLUPS"], 3)
        out["aa_layout"] = {st: timed_run(wl, st, n, warm, dev) for st in ("f16s", "bf16s")}
        return out

    out = study(W.workload("rotor1024_q27"), "rotor1024_q27: 512x512x1024 D3Q27, R=128 NACA4412 rotor, TSR 7",
                steps, 5)
    out["d3q19"] = study(W.workload("rotor256"),
                         "rotor256: 256x256x512 D3Q19, R=64 NACA4412 rotor, TSR 6, 5% turbulence",
                         max(steps, 200), 10)
    return out


def farm_run(dev, steps):
    """Wind-farm scale on one GPU: 1536x512x1024 D3Q19 FP32, 3x2 rotors R=64."""
    import workloads as W
    wl = W.workload("farm")
    r = timed_run(wl, "f32", steps, 5, dev)
    r["workload"] = "farm: 1536x512x1024 (805M cells) D3Q19 FP32, 6 rotors R=64, flow along x, 5% turbulence"
    return r


def farm_wake(dev, steps, sample_every=50):
    """Wind farm: per-rotor mean thrust and torque over the second half of
    `steps` steps, and the time-averaged axial velocity there on lateral lines
    (along z at hub height, +-1.5 D around the rotor centre, every D/8) 2 D and
    4 D downstream of each rotor (D = 2 R)."""
    import torch
    import workloads as W
    from paper_2510_13726_b300 import Lattice
    wl = W.workload("farm")
    lat = Lattice.from_workload(wl, device=dev)
    half = steps // 2
    lat.step(half)
    lat.forces(reset_avg=True)
    lines = []
    for r in wl.rotors:
        D = 2.0 * r.radius
        cx, cy, cz = (int(round(v)) for v in r.center)
        zs = [int(round(cz + k * D / 8)) for k in range(-12, 13)]
        zs = [z for z in zs if 0 <= z < wl.nz]
        xs = [int(round(cx + m * D)) for m in (2, 4)]
        lines.append((cy, zs, xs))
    acc = [torch.zeros(2, len(zs), dtype=torch.float64, device=dev) for (_, zs, _) in lines]
    n = 0
    done = 0
    while done < steps - half:
        k = min(sample_every, steps - half - done)
        lat.step(k)
        done += k
        _, u = lat.fields()
        for a, (cy, zs, xs) in zip(acc, lines):
            zi = torch.tensor(zs, device=dev)
            for j, x in enumerate(xs):
                if 0 <= x < wl.nx:
                    a[j] += u[0].index_select(0, zi)[:, cy, x].double()
        n += 1
        del u
    _, Fa = lat.forces()
    _, Ma = lat.moments()
    out = {"workload": "farm: 1536x512x1024 D3Q19 FP32, 6 rotors R=64, flow along x, 5% turbulence",
           "steps": steps, "averaged_steps": steps - half, "samples": n, "u_in": wl.u_in, "rotors": []}
    for i, ((cy, zs, xs), a) in enumerate(zip(lines, acc)):
        r = wl.rotors[i]
        prof = (a / max(1, n)).cpu().numpy()
        out["rotors"].append({
            "center": [round(v, 2) for v in r.center], "thrust_mean": round(float(Fa[i, 0]), 6),
            "torque_mean": round(float(Ma[i, 0]), 6), "z_offsets_D": [round((z - r.center[2]) / (2 * r.radius), 3) for z in zs],
            "u_axial_2D": [round(float(v), 5) for v in prof[0]] if 0 <= xs[0] < wl.nx else None,
            "u_axial_4D": [round(float(v), 5) for v in prof[1]] if 0 <= xs[1] < wl.nx else None})
    lat.close()
    del lat
    torch.cuda.empty_cache()
    return out


def driven_run(dev, steps):
    """rotor256 with the rotor turning under its own torque and a generator
    law (evolve structure on the device) against the same steps prescribed."""
    import torch
    import workloads as W
    from paper_2510_13726_b300 import Lattice
    wl = W.workload("rotor256")
    om0 = wl.rotors[0].omega(wl.u_in)
    out = {"workload": "rotor256 with a torque-driven rotor (I = 1e6, generator k = 2e3)", "steps": steps}
    for mode in ("prescribed", "driven"):
        lat = Lattice.from_workload(wl, device=dev)
        lat.step(5)
        if mode == "driven":
            lat.set_drive(0, 1e6, k_gen=2e3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(lat.stream)
        lat.step_async(steps)
        e1.record(lat.stream)
        e1.synchronize()
        lat.check()
        ms = e0.elapsed_time(e1) / steps
        th, om = lat.drive_state(0)
        out[mode] = {"MLUPS": round(wl.cells / ms / 1e3, 1), "ms_per_step": round(ms, 4),
                     "omega_start": om0, "omega_end": om}
        lat.close()
        del lat
        torch.cuda.empty_cache()
    return out


def adjoint_run(dev, steps, avg_last, ckpt_every):
    """Gradient of the time-averaged thrust on the 128x128x256 D3Q19 rotor
    (R = 32): hl_grad over `steps` steps (checkpoint every `ckpt_every`)
    against the same number of plain forward steps from the same state."""
    import torch
    import workloads as W
    from paper_2510_13726_b300 import Lattice
    wl = W.workload("rotor128_adj")
    lat = Lattice.from_workload(wl, device=dev)
    lat.step(5)
    state = lat.save_state()
    nb = lat.grad_workspace_size(steps, ckpt_every)
    work = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
    work = work[(-work.data_ptr()) % 256:]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(lat.stream)
    lat.step_async(steps)
    e1.record(lat.stream)
    e1.synchronize()
    lat.check()
    fwd = e0.elapsed_time(e1) / steps
    lat.load_state(state)
    torch.cuda.synchronize(dev)
    e0.record(lat.stream)
    J, gp, gd = lat.grad(steps, avg_last, [1.0], [0.0], ckpt_every=ckpt_every, work=work)
    e1.record(lat.stream)
    e1.synchronize()
    grad = e0.elapsed_time(e1) / steps
    finite = bool(torch.isfinite(gd).all().item())
    lat.close()
    del lat, work, gd
    torch.cuda.empty_cache()
    return {"workload": "rotor128_adj: 128x128x256 D3Q19 FP32, R=32 NACA4412 rotor, TSR 6",
            "objective": f"mean thrust over the last {avg_last} of {steps} steps",
            "steps": steps, "ckpt_every": ckpt_every, "workspace_gb": round(nb / 1e9, 2),
            "forward_ms_per_step": round(fwd, 4), "grad_ms_per_step": round(grad, 4),
            "ratio_end_to_end": round(grad / fwd, 3),
            "reverse_ms_per_step": round(grad - fwd, 4),
            "ratio_reverse_per_step": round((grad - fwd) / fwd, 3),
            "J": J, "dJ_dpitch": float(gp[0]), "dJ_dd0_finite": finite}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", default="rotor256")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16s", "bf16s"])
    ap.add_argument("--layout", default="aa", choices=["aa", "esotwist", "aa_halves"],
                    help="population layout: AA pattern, esoteric twist, or AA pattern with x halves")
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 16-bit storage study, the farm run and the gradient run")
    ap.add_argument("--extras", default="storage,farm,adjoint,driven",
                    help="comma-separated extra studies after the main line: storage, farm, adjoint, driven")
    ap.add_argument("--extra-steps", type=int, default=40)
    ap.add_argument("--farm-wake-steps", type=int, default=0,
                    help="steps of the wind-farm wake study (mean loads and axial-velocity lines 2 D and 4 D "
                         "behind each rotor over the second half); 0 skips it")
    ap.add_argument("--adjoint-steps", type=int, default=4000,
                    help="steps of the gradient run (config of the adjoint/forward ratio); 0 skips it")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "cuda":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_cuda(args)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Throughput of the fused collide-and-stream update of the vectorial D2Q5 scheme.

Workload (one GPU): periodic double shear layer on a 4096^2 lattice, 3 fields x
5 velocities = 15 populations per node stored in FP32 (deviations from the rest
equilibrium), nu = 1e-4, mu = 8, omega_rho = 6/5, alpha_rho = 3/40,
omega_q = 23/20 (Section 6.1 defaults), synthetic seeded input.  One step = one
lattice update of every node (relaxation + transport).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vlbm|reference]

--impl reference times the FP64 CPU oracle (test infrastructure, as it stands)
on the same workload on the host cores, each step one full-lattice update,
bounded in total time.  Under torchrun (N > 1) each rank advances its own
independent replica of the lattice (no data-path collective); the elapsed time
is the max over ranks.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % HBM roofline; time-to-t at stated L2 error vs plain FP32 LBM"
UNIT = "GLUPS"
ELEM_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2, "fp16split": 2, "bf16split": 2}
CTYPE = {"fp64": "double", "fp32": "float", "fp16": "__half", "bf16": "__nv_bfloat16", "fp16split": "__half",
         "bf16split": "__nv_bfloat16"}
WORKLOADS = {
    # name: (dim, populations per node, default side, nu)
    "dsl2d": (2, 15, 4096, 1e-4),
    "tgv3d": (3, 28, 256, 1.0 / 1600.0),
    "batch512": (2, 15, 0, None),      # 512 problems: sides and nu drawn per problem
    "sur256": (2, 15, 1024, 1e-3),     # learned surrogate on 256^2, pooled from 1024^2 runs
    "poiseuille": (2, 15, 253, 1e-2),  # channel of Section 6.2 (Table 2), 75..253 cells per direction
}

# Table 2 of the paper (Section 6.2.2): L2 error on u_x at t = 0.05, omega_rho = 6/5, alpha_rho = 3/40;
# (cells, omega_q, wall correction) -> printed value
TABLE2 = {
    (75, 1.0, False): 2.938e-05, (112, 1.0, False): 1.333e-05, (168, 1.0, False): 5.994e-06, (253, 1.0, False): 2.668e-06,
    (75, 1.15, False): 5.661e-04, (112, 1.15, False): 3.812e-04, (168, 1.15, False): 2.563e-04, (253, 1.15, False): 1.707e-04,
    (75, 1.0, True): 2.943e-05, (112, 1.0, True): 1.335e-05, (168, 1.0, True): 5.997e-06, (253, 1.0, True): 2.670e-06,
    (75, 1.15, True): 1.485e-05, (112, 1.15, True): 6.672e-06, (168, 1.15, True): 3.043e-06, (253, 1.15, True): 1.368e-06,
}


def split(args):
    return args.precision.endswith("split")


def bytes_per_node(args):
    """Algorithmic bytes of one node update: every stored value read once and written once
    (split layouts: one FP32 moment per field and 16-bit non-equilibrium parts of the moving
    populations)."""
    dim, ppn = WORKLOADS[args.workload][:2]
    if split(args):
        fields = dim + 1
        return 2 * (fields * 4 + (ppn - fields) * 2)
    return 2 * ppn * ELEM_BYTES[args.precision]


def kernel_name(args):
    dim = WORKLOADS[args.workload][0]
    if split(args):
        lanes = (args.split_lanes or 4) if dim == 2 else None
        mid = f", {lanes}" if lanes else ""
        return f"k_split_step_{dim}d_vec<{CTYPE[args.precision]}{mid}, false>"
    return f"k_stream_collide_{dim}d_vec<{CTYPE[args.precision]}, false, false>"
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["vlbm", "reference"], default="vlbm")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="dsl2d")
    ap.add_argument("--n", type=int, default=None, help="lattice side (default: 4096 in 2D, 256 in 3D)")
    ap.add_argument("--precision", choices=list(ELEM_BYTES), default="fp32")
    ap.add_argument("--count", type=int, default=512, help="problems of the batch512 workload")
    ap.add_argument("--batch-launch", choices=["persistent", "graph"], default="persistent",
                    help="batch512: all timed steps in one cooperative launch (persistent), or one launch per "
                         "step replayed from 32-step CUDA graphs")
    ap.add_argument("--split-lanes", type=int, choices=[2, 4], default=None,
                    help="nodes per lane of the 2D split kernels (tuning)")
    ap.add_argument("--kernel", type=int, choices=[0, 1, 2], default=0,
                    help="VLBM_OPT_KERNEL of the lattice: 0 automatic, 1 per node, 2 vectorised")
    ap.add_argument("--sur-trajectories", type=int, default=200, help="sur256: training trajectories (100 pairs each)")
    ap.add_argument("--sur-epochs", type=float, default=8.0, help="sur256: training epochs")
    ap.add_argument("--sur-batch", type=int, default=32, help="sur256: states advanced together in the timed rollouts")
    ap.add_argument("--sur-k", type=int, default=32,
                    help="sur256: fine lattice steps per surrogate step (a multiple of 16); the rollout covers "
                         "3200 fine steps (3072 for K = 256)")
    ap.add_argument("--conv-only", action="store_true",
                    help="sur256: time only the dominant kernel (the 64 -> 64 conv of the rollout) and the "
                         "training step's weight gradient of that conv, no training")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-history", action="store_true", help="tgv3d: skip the energy and dissipation history")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--cpu-seconds-one-core", type=float, default=8.0,
                    help="target CPU time of the single-threaded oracle sample")
    ap.add_argument("--reference-seconds", type=float, default=150.0, help="cap on the reference arm's timed steps")
    args = ap.parse_args()
    if args.n is None:
        args.n = WORKLOADS[args.workload][2]
    if args.workload == "sur256":
        if "--steps" not in sys.argv:
            args.steps = 10
        if "--warmup" not in sys.argv:
            args.warmup = 3
    if args.workload == "batch512" and args.precision == "fp32" and "--precision" not in sys.argv:
        args.precision = "fp16split"     # the batched workload stores 16-bit populations by default
    return args


def nodes_of(args):
    return args.n ** WORKLOADS[args.workload][0]


def make_input(args):
    """(u, phi, dx, n-tuple) of the workload; seeded and synthetic."""
    import synthetic
    if args.workload == "dsl2d":
        u, phi, dx = synthetic.double_shear_layer(args.n)
        return u, phi, dx, (args.n, args.n)
    u, phi, dx = synthetic.taylor_green_3d(args.n)
    return u, phi, dx, (args.n,) * 3


def workload_config(args, extra=None):
    dim, ppn, _, nu = WORKLOADS[args.workload]
    if args.workload == "dsl2d":
        name = f"double shear layer {args.n}x{args.n} periodic, D2Q5 vectorial (3 fields x 5 velocities)"
        init = "u_x = tanh(80(y - pi/2)) (y <= pi) / tanh(80(3pi/2 - y)), u_y = 0.05 sin x, phi = 0"
    else:
        name = f"Taylor-Green vortex {args.n}^3 periodic, D3Q7 vectorial (4 fields x 7 velocities)"
        init = "u = (sin x cos y cos z, -cos x sin y cos z, 0), phi = (cos 2x + cos 2y)(cos 2z + 2)/16"
    cfg = {
        "workload": name,
        "lattice": [args.n] * dim,
        "populations_per_node": ppn,
        "storage": args.precision,
        "nu": nu, "mu": 8.0, "omega_rho": 1.2, "alpha_rho": 0.075, "omega_q": 1.15,
        "init": init,
        "l2": l2_note(nodes_of(args) * bytes_per_node(args) / 2),
    }
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------- distributed plumbing
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
        return dist
    return None


def max_over_ranks(value, dist, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.buf = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.buf, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.buf = ""

    def summary(self):
        if not self.buf:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        rows = [r for r in csv.reader(io.StringIO(self.buf)) if len(r) >= 9]
        sm = []
        sm_max = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                sm_max = float(r[2])
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        loaded = [s for s in sm if sm_max and s > 0.3 * sm_max] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": sm_max,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline inputs
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# sources that define the stream-collide step kernels (the surrogate's and the
# no-allocation entry's files do not change them)
# Sources each step kernel is compiled from (its code and its launch shape): a profiled figure stays
# valid while these files are unchanged.
STEP_SOURCES = {
    "2d": ("vlbm_device.cuh", "vlbm_kernels_2d.cuh", "vlbm_api.cu", "vlbm_host.hpp"),
    "3d": ("vlbm_device.cuh", "vlbm_kernels_2d.cuh", "vlbm_kernels_3d.cuh", "vlbm_api.cu", "vlbm_host.hpp"),
    "split": ("vlbm_device.cuh", "vlbm_kernels_2d.cuh", "vlbm_kernels_3d.cuh", "vlbm_split.cuh", "vlbm_api.cu",
              "vlbm_host.hpp"),
    "batch": ("vlbm_device.cuh", "vlbm_kernels_2d.cuh", "vlbm_kernels_3d.cuh", "vlbm_split.cuh", "vlbm_batch.cu",
              "vlbm_host.hpp"),
}


def source_kind(args):
    if args.workload == "batch512":
        return "batch"
    if split(args):
        return "split"
    return "3d" if WORKLOADS[args.workload][0] == 3 else "2d"


def l2_note(lattice_bytes: float) -> str:
    """The timing-hygiene note of a run: two lattice copies above the 126 MB L2 need no flush."""
    if 2 * lattice_bytes > 126e6:
        return "working set 2 lattices x {:.2f} GB > 126 MB L2: no flush needed".format(lattice_bytes / 1e9)
    return "working set 2 lattices x {:.1f} MB fits in the 126 MB L2 (a small case)".format(lattice_bytes / 1e6)


def source_digest(kind):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2607_24059_b300", "csrc")
    for fn in STEP_SOURCES[kind]:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, n, digest):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    for e in d.get("entries", []):
        if e.get("kernel") == kernel and e.get("source_digest") == digest and e.get("n") == n:
            return float(e["dram_bytes_per_launch"])
    return None


# ---------------------------------------------------------------- CPU oracle baseline
def oracle_sample(args, seconds, threads=None):
    """GLUPS of the FP64 oracle on the same lattice, on the host cores, for ~seconds
    (threads: OpenMP threads, default all)."""
    import oracle
    import synthetic
    orc = oracle.default()
    all_threads = orc.num_threads()
    if threads:
        orc.set_num_threads(threads)
    try:
        u, phi, dx, n = make_input(args)
        p = oracle.make_params(n, dx, nu=WORKLOADS[args.workload][3])
        f = orc.init(p, u, phi)
        work = np.empty_like(f)
        warm = 1 if threads == 1 else 2
        orc.run_inplace(p, f, work, warm)     # warm-up (first touch of the work lattice, thread start)
        m = 0
        t0 = time.perf_counter()
        while True:                           # whole steps until the time budget is used
            orc.run_inplace(p, f, work, 1)
            m += 1
            el = time.perf_counter() - t0
            if el >= seconds or m >= 500:
                break
        cores = orc.num_threads()
    finally:
        orc.set_num_threads(all_threads)
    return {"value": nodes_of(args) * m / el / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{args.workload} {args.n}^{WORKLOADS[args.workload][0]}, {m} FP64 oracle steps after {warm} "
                      f"warm-up step(s) (plain C, OpenMP over rows, {cores} thread(s))", "seconds": el}


def tgv3d_history(lat, u, phi, nu, steps, every, torch):
    """Kinetic energy E(t) and the dissipation of the 3D Taylor-Green vortex every `every` steps
    over `steps` steps (both FP64 reductions on the GPU): -dE/dt from centred differences of the
    E history against nu * sum |curl u|^2 dx^3 (centred differences of the velocity)."""
    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    dt = lat.derived.dt
    t, e, eps = [], [], []
    for j in range(steps // every + 1):
        if j:
            lat.step(every)
        t.append(lat.time()[1])
        e.append(float(lat.invariants()[4]))
        eps.append(nu * lat.vorticity_sq())
    t, e, eps = np.array(t), np.array(e), np.array(eps)
    dEdt = -(e[2:] - e[:-2]) / (t[2:] - t[:-2])
    mism = np.abs(dEdt - eps[1:-1]) / np.abs(eps[1:-1])
    pick = np.linspace(0, len(t) - 1, 11).round().astype(int)
    return {"steps": steps, "every": every, "dt": dt, "reduction": "FP64 on the GPU (vlbm_invariants, vlbm_vorticity_sq)",
            "E0": e[0], "E_end": e[-1], "t_end": t[-1],
            "dissipation_vs_minus_dEdt_max_rel_diff": float(mism.max()),
            "dissipation_vs_minus_dEdt_mean_rel_diff": float(mism.mean()),
            "samples": {"t": [float(t[i]) for i in pick], "E": [float(e[i]) for i in pick],
                        "nu_curl_sq": [float(eps[i]) for i in pick],
                        "minus_dEdt": [float(dEdt[min(max(i - 1, 0), len(dEdt) - 1)]) for i in pick]}}


# ---------------------------------------------------------------- the two arms
def run_reference_poiseuille(args):
    """Reference arm of the channel workload: the oracle's Poiseuille simulation (ghost-cell
    boundaries of Section 6.2.1) on the host cores, the 75-cell row of Table 2 (four runs)."""
    import oracle
    from oracle.poiseuille import Poiseuille
    orc = oracle.default()
    rows, nodes, t0 = [], 0, time.perf_counter()
    for omega_q in (1.0, 1.15):
        for corrected in (False, True):
            sim = Poiseuille(orc, 75, omega_q, corrected=corrected)
            steps = sim.run_to(0.05)
            nodes += 75 * 75 * steps
            rows.append({"cells": 75, "omega_q": omega_q, "wall_correction": corrected, "steps": steps,
                         "l2_error_ux": sim.l2_error_ux(), "table2": TABLE2[(75, omega_q, corrected)]})
    el = time.perf_counter() - t0
    value = nodes / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": rows[0]["steps"],
        "warmup": 0, "ms_per_step": el / (4 * rows[0]["steps"]) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "Poiseuille channel of Section 6.2 (Table 2), 75-cell row", "storage": "fp64 (oracle)"},
        "table2": rows,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                         "sample": "the four 75-cell runs of Table 2 to t = 0.05 (2250 steps each)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "poiseuille":
        return run_reference_poiseuille(args)
    if args.workload not in ("dsl2d", "tgv3d"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times the single-lattice workloads "
                          f"(dsl2d, tgv3d) and the channel; {args.workload} has no oracle arm"}), flush=True)
        return 0
    import oracle
    import synthetic
    orc = oracle.default()
    u, phi, dx, n = make_input(args)
    p = oracle.make_params(n, dx, nu=WORKLOADS[args.workload][3])
    f = orc.init(p, u, phi)
    work = np.empty_like(f)
    orc.run_inplace(p, f, work, max(1, min(args.warmup, 3)))
    done = 0
    t0 = time.perf_counter()
    while done < args.steps:
        orc.run_inplace(p, f, work, 1)
        done += 1
        if time.perf_counter() - t0 > args.reference_seconds:
            break
    el = time.perf_counter() - t0
    value = nodes_of(args) * done / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": done,
        "steps_requested": args.steps, "warmup": max(1, min(args.warmup, 3)), "ms_per_step": el / done * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, {"storage": "fp64 (oracle)"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                         "sample": f"{done} full-lattice FP64 oracle steps (capped at {args.reference_seconds:.0f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_vlbm(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, "nccl")
    import paper_2607_24059_b300 as vlbm
    import synthetic

    u, phi, dx, shape = make_input(args)
    lat = vlbm.Lattice(shape, dx, nu=WORKLOADS[args.workload][3], precision=args.precision)
    if args.split_lanes:
        lat.set_option(vlbm.VLBM_OPT_SPLIT_LANES, args.split_lanes)
    if args.kernel:
        lat.set_option(vlbm.VLBM_OPT_KERNEL, args.kernel)
    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    # warm-up: W steps, then prime the captured step graphs (64, 16 and 4 steps) of both
    # buffer parities, so that no capture happens inside the timed region
    lat.step(args.warmup)
    for _ in range(2):
        for k in (64, 16, 4, 1):
            lat.step(k)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    # ---- device-resident timing (inputs already in HBM)
    c0 = lat.launch_count()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        lat.step(args.steps)
        end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = start.elapsed_time(end) / 1e3
    launches = lat.launch_count() - c0
    elapsed_max = max_over_ranks(elapsed, dist, "cuda")
    nodes = nodes_of(args)
    value = world * nodes * args.steps / elapsed_max / 1e9
    inv = lat.invariants()
    assert inv[6] == 0, "non-finite populations after the timed steps"

    # roofline of the stream-collide kernel (the only kernel in the timed region)
    per_launch = elapsed / args.steps
    bpn = bytes_per_node(args)
    achieved = bpn * nodes / per_launch / 1e9
    peak, peak_kind = measured_peaks()
    digest = source_digest(source_kind(args))
    traffic = profiled_traffic(kernel_name(args), args.n, digest)

    # ---- end to end through the C ABI with host buffers
    u_host = torch.from_numpy(u.astype(np.float32)).pin_memory()
    # a workload whose initial potential is zero (the shear layer) passes none: vlbm_init takes
    # a null phi as phi = 0, so only the velocity crosses the bus
    phi_host = torch.from_numpy(phi.astype(np.float32)).pin_memory() if np.any(phi) else None
    u_out = torch.empty_like(u_host).pin_memory()
    hist = torch.zeros((args.steps, 8), dtype=torch.float64).pin_memory()
    # warm-up of the same path (first use of the recorded-step and read-back kernels), untimed
    vlbm.vlbm_init(lat.handle, u_host, phi_host)
    for s in range(max(args.warmup, 3)):
        vlbm.vlbm_step_record(lat.handle, 1, 1, hist[s % args.steps])
    vlbm.vlbm_macros(lat.handle, None, u_out, None)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vlbm.vlbm_init(lat.handle, u_host, phi_host)             # H2D of the step's input
    for s in range(args.steps):
        vlbm.vlbm_step_record(lat.handle, 1, 1, hist[s])     # step + fused invariants, D2H of 64 B
    vlbm.vlbm_macros(lat.handle, None, u_out, None)          # D2H of the velocity field
    torch.cuda.synchronize()
    e2e_el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = world * nodes * args.steps / e2e_el / 1e9
    assert np.all(np.isfinite(hist.numpy())) and np.all(np.isfinite(u_out.numpy()))
    ubytes = u_host.numel() * u_host.element_size()
    pbytes = 0 if phi_host is None else phi_host.numel() * phi_host.element_size()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64"}.get(args.precision, args.precision + "-storage/f32"),
        "data": "synthetic",
        "config": workload_config(args, {"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                         "graph_prime_steps": 170}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic, "bytes_per_node": bpn,
                     "kernel": kernel_name(args), "avg_launch_ms": per_launch * 1e3,
                     "source_digest": digest},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": (ubytes + pbytes) / args.steps,
                "d2h_bytes_per_step": 64 + ubytes / args.steps,
                "how": ("vlbm_init from pinned host u" + (" and phi" if phi_host is not None else
                        " (phi = 0: none passed)")) + ", per step vlbm_step_record (fused invariants: 64 B "
                       "D2H per step, written by the step kernel into the mapped pinned record buffer), vlbm_macros "
                       "to pinned host u; untimed warm-up of the same calls first"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if args.workload == "tgv3d" and world == 1 and not args.no_history:
        line["history"] = tgv3d_history(lat, u, phi, WORKLOADS["tgv3d"][3], 2000, 10, torch)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(args, args.cpu_seconds)
        one = oracle_sample(args, args.cpu_seconds_one_core, threads=1)
        line["cpu_baseline"]["one_core"] = {"value": one["value"], "unit": UNIT, "cores": one["cores"],
                                            "sample": one["sample"]}
    print(json.dumps(line), flush=True)
    lat.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """512 independent periodic problems (sides 64..1024, nu log-uniform in [1e-4, 1e-2],
    divergence-free random Fourier initial fields), one launch per step, autotuned."""
    import torch
    import paper_2607_24059_b300 as vlbm
    import synthetic
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    count = args.count
    probs = synthetic.batched_problem_set(count)
    specs, inputs = [], []
    for q in probs:
        u, phi, dx = synthetic.random_fourier_field(q.side, q.seed)
        specs.append(dict(n=(q.side, q.side), dx=dx, nu=q.nu))
        inputs.append((u.astype(np.float32), phi.astype(np.float32)))
    b = vlbm.Batch(specs, precision=args.precision)
    nodes = sum(q.side * q.side for q in probs)
    t0 = time.perf_counter()
    for i, (u, phi) in enumerate(inputs):
        b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    torch.cuda.synchronize()
    cfg, tuned_ms = b.autotune(repeats=3)
    b.step(args.warmup)
    b.step(64)
    b.step(1)
    b.step(64)
    persistent = args.batch_launch == "persistent"
    if persistent:
        b.step(max(args.warmup, 3), persistent=True)
    torch.cuda.synchronize()
    launches0 = b.info()[2]
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record(stream)
        b.step(args.steps, persistent=persistent)
        end.record(stream)
        torch.cuda.synchronize()
    elapsed = start.elapsed_time(end) / 1e3
    launches = b.info()[2] - launches0
    # e2e: initial fields from pinned host memory, the steps, every velocity field back to pinned host
    pinned = [(torch.from_numpy(u).pin_memory(), torch.from_numpy(phi).pin_memory()) for u, phi in inputs]
    outs = [torch.empty_like(u) .pin_memory() for u, _ in pinned]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (u, phi) in enumerate(pinned):
        vlbm.vlbm_batch_init(b.handle, i, u, phi)
    b.step(args.steps, persistent=persistent)
    for i, o in enumerate(outs):
        vlbm.vlbm_batch_macros(b.handle, i, None, o, None)
    torch.cuda.synchronize()
    e2e_el = time.perf_counter() - t0
    # the scheme itself diverges on the set's under-resolved problems (small sides, low nu: the
    # FP64 oracle does too), so the count of non-finite fields is reported, not asserted
    nonfinite = [i for i, o in enumerate(outs) if not bool(torch.isfinite(o).all())]
    in_bytes = sum(u.numel() * 4 + phi.numel() * 4 for u, phi in pinned)
    out_bytes = sum(o.numel() * 4 for o in outs)
    bpn = bytes_per_node(args)
    achieved = bpn * nodes / (elapsed / args.steps) / 1e9
    peak, peak_kind = measured_peaks()
    kname = "{}<{}, {}>".format("k_batch_steps_2d" if persistent else "k_batch_step_2d", CTYPE[args.precision],
                                "split" if split(args) else "uniform")
    digest = source_digest("batch")
    # DRAM bytes of one step of the whole batch (a persistent launch runs several steps)
    traffic = profiled_traffic(kname, count, digest)
    line = {
        "metric": METRIC, "value": nodes * args.steps / elapsed / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64"}.get(args.precision, args.precision + "-storage/f32"),
        "data": "synthetic",
        "config": {"workload": f"{count} independent periodic 2D problems, sides 64..1024, nu 1e-4..1e-2, "
                               "random Fourier initial fields", "nodes": nodes, "storage": args.precision,
                   "autotuned": {"threads": cfg[0], "blocks_per_sm": cfg[1], "lanes": cfg[2],
                                 "ms_per_step": tuned_ms},
                   "launch": ("all timed steps in one cooperative launch, grid barrier between steps"
                              if persistent else "one launch per step, replayed from 32-step CUDA graphs"),
                   "l2": l2_note(nodes * bpn / 2),
                   "nonfinite_after_steps": {"problems": len(nonfinite), "steps": args.steps,
                                             "note": "under-resolved problems diverge in the scheme itself "
                                                     "(the FP64 oracle as well); the work per node is the same"}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic, "bytes_per_node": bpn, "kernel": kname,
                     "avg_launch_ms": elapsed / args.steps * 1e3, "per": "one step of every problem",
                     "source_digest": digest},
        "e2e": {"value": nodes * args.steps / e2e_el / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": in_bytes / args.steps, "d2h_bytes_per_step": out_bytes / args.steps},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def conv_roofline(nb, c, stream, reps=50):
    """The rollout's dominant kernel, the 64 -> 64 periodic 3x3 conv with GELU on nb states of
    c^2 pixels, timed alone with CUDA events (reps launches after 3 warm-up launches)."""
    import torch
    import paper_2607_24059_b300 as vlbm
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(7)
    X = torch.randn(nb, c, c, 64, device="cuda", generator=g).to(torch.bfloat16)
    Wt = (0.05 * torch.randn(64, 9, 64, device="cuda", generator=g)).to(torch.bfloat16)
    bias = torch.zeros(64, device="cuda")
    Yc = torch.empty_like(X)
    for _ in range(3):
        vlbm.vlbm_sur_conv3x3(X, Wt, bias, Yc, err, act=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        vlbm.vlbm_sur_conv3x3(X, Wt, bias, Yc, err, act=True)
    e1.record(stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    conv_ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * nb * c * c * 9 * 64 * 64
    peaks = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            peaks = json.load(fh)
    peak = float(peaks.get("bf16_tflops", 1800.0))
    achieved = flops / (conv_ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_kind": "measured (cuBLAS bf16 burst)" if "bf16_tflops" in peaks else "fallback",
            "traffic": None, "kernel": "k_conv3x3<64, 64, true, false>", "avg_launch_ms": conv_ms,
            "flops_per_launch": flops, "launches_timed": reps,
            "algorithmic_bytes_per_launch": nb * c * c * 64 * 2 * 2}


def wgrad_roofline(nb, c, stream, reps=20):
    """The training step's largest kernel, the weight and bias gradients of the 64 -> 64 conv on nb
    states of c^2 pixels, timed alone with CUDA events (reps launches after 3 warm-up launches)."""
    import torch
    import paper_2607_24059_b300 as vlbm
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(8)
    X = torch.randn(nb, c, c, 64, device="cuda", generator=g).to(torch.bfloat16)
    dZ = torch.randn(nb, c, c, 64, device="cuda", generator=g).to(torch.bfloat16)
    G = torch.zeros(64, 9, 64, device="cuda")
    Gb = torch.zeros(64, device="cuda")
    for _ in range(3):
        vlbm.vlbm_sur_conv3x3_wgrad(X, dZ, G, Gb, err)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        vlbm.vlbm_sur_conv3x3_wgrad(X, dZ, G, Gb, err)
    e1.record(stream)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * nb * c * c * 9 * 64 * 64
    return {"kernel": "k_conv3x3_wgrad<64, 64>", "avg_launch_ms": ms, "flops_per_launch": flops,
            "achieved_tflops": flops / (ms * 1e-3) / 1e12, "launches_timed": reps}


def run_surrogate(args):
    """Learned surrogate (256^2 states pooled 4x from 1024^2 runs of the scheme; u_x, u_y, phi):
    one step of this workload is a checked rollout of --sur-batch states by 100 surrogate steps
    (100 x 32 fine lattice steps).  value = time-to-t speedup per state over the plain FP32
    scheme on the 1024^2 lattice on the same GPU, at the L2 velocity error stated in config."""
    import torch
    import paper_2607_24059_b300 as vlbm
    from paper_2607_24059_b300 import surrogate as sg
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if args.conv_only:
        if rank == 0:
            stream = torch.cuda.current_stream()
            print(json.dumps({"workload": "sur256 dominant kernel alone", "states": args.sur_batch,
                              "roofline": conv_roofline(args.sur_batch, args.n // 4, stream),
                              "wgrad": wgrad_roofline(args.sur_batch, args.n // 4, stream)}), flush=True)
        return 0
    dist = dist_init(world, "nccl")
    cfg = sg.Config(fine=args.n, train_trajectories=args.sur_trajectories, epochs=args.sur_epochs,
                    k_fine=args.sur_k, rollout_steps=max(1, 3200 // args.sur_k))
    tr = sg.train_surrogate(cfg, log=lambda m: print(m, file=sys.stderr, flush=True))
    net, nb, steps = tr.net, args.sur_batch, cfg.rollout_steps
    ref = tr.test_snaps.transpose(0, 1).contiguous()              # (steps + 1, states, C, c, c)
    ntest = ref.shape[1]
    ro = sg.Rollout(net, cfg, max(nb, ntest), div_limit=tr.div_limit)
    # accuracy against the fine scheme, checked and unchecked
    _, acc = ro.run(ref[0].contiguous(), steps, check=True, reference=ref, every=steps)
    _, acc_free = ro.run(ref[0].contiguous(), steps, check=False, reference=ref, every=steps)
    _, coarse_err = sg.coarse_scheme(cfg, ref[0].contiguous(), steps, reference=ref[-1])
    t_fine = sg.fine_time_to_t(cfg, cfg.test_seeds()[0])
    u0 = ref[0][torch.arange(nb) % ntest].contiguous()
    for _ in range(max(args.warmup, 3)):
        ro.run(u0, steps)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    l0, c0 = vlbm.vlbm_sur_launch_count(), ro.coarse.info()[2]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fallbacks = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            _, info = ro.run(u0, steps)
            fallbacks += sum(info["fallbacks"])
        end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = max_over_ranks(start.elapsed_time(end) / 1e3, dist, "cuda")
    launches = (vlbm.vlbm_sur_launch_count() - l0) + (ro.coarse.info()[2] - c0)
    ms_per_state = elapsed / args.steps / nb * 1e3
    value = world * t_fine / ms_per_state
    # end to end: states from pinned host memory, the checked rollout, states back to pinned host
    h_in = u0.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty_like(u0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        d_in.copy_(h_in, non_blocking=True)
        out, _ = ro.run(d_in, steps)
        h_out.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e2e_el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = world * t_fine / (e2e_el / args.steps / nb * 1e3)
    c = cfg.coarse
    roof = conv_roofline(nb, c, stream)
    ro.close()
    # the plain scheme on the coarse lattice with the same batching (nb states, one launch per step)
    cb = vlbm.Batch([dict(n=(c, c), dx=2 * math.pi / c, nu=cfg.nu)] * nb, precision="fp32")
    mask = torch.ones(nb, dtype=torch.uint8, device=u0.device)
    outs = torch.empty_like(u0)

    def coarse_batch_run():
        vlbm.vlbm_batch_init_states(cb.handle, u0, mask)
        cb.step(steps * cfg.coarse_steps)
        vlbm.vlbm_batch_macros_states(cb.handle, outs, mask)
    coarse_batch_run()
    c0e, c1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0e.record(stream)
    for _ in range(args.steps):
        coarse_batch_run()
    c1e.record(stream)
    torch.cuda.synchronize()
    coarse_ms_per_state = c0e.elapsed_time(c1e) / args.steps / nb
    cb.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "x time-to-t speedup per state vs plain FP32 LBM 1024^2",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (FP32 accumulate)", "data": "synthetic (scheme-generated)",
        "config": {
            "workload": f"learned surrogate: 5 periodic 3x3 convs (64 ch, GELU) on {c}^2 states (u_x, u_y, phi) "
                        f"pooled {cfg.factor}x from {cfg.fine}^2 FP32 runs of the scheme, nu = {cfg.nu}; "
                        f"{steps} surrogate steps of {cfg.k_fine} fine steps each, checked (energy, divergence) "
                        "with the plain coarse-lattice scheme as fallback",
            "states_per_step": nb, "training_pairs": cfg.train_trajectories * cfg.pairs_per_trajectory,
            "train_seconds": tr.summary["seconds"], "train_steps": tr.summary["steps"],
            "l2_rel_error_checked": acc["curve"][-1][1], "l2_rel_error_unchecked": acc_free["curve"][-1][1],
            "l2_rel_error_coarse_scheme": float(np.mean(coarse_err)),
            "fallbacks_per_state_step": fallbacks / (args.steps * nb * steps),
            "fine_fp32_ms_per_state": t_fine, "surrogate_ms_per_state": ms_per_state,
            "coarse_fp32_ms_per_state_same_batching": coarse_ms_per_state,
            "coarse_scheme_speedup_same_batching": t_fine / coarse_ms_per_state,
            "l2": "rollout states 32 x 3 x 256^2 FP32 = 25 MB (L2-resident, as in use)"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "x time-to-t speedup per state vs plain FP32 LBM 1024^2",
                "h2d_bytes_per_step": h_in.numel() * 4, "d2h_bytes_per_step": h_out.numel() * 4},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    net.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_poiseuille(args):
    """The channel test of Section 6.2 on the GPU: every row of Table 2 (75, 112, 168, 253 cells,
    omega_q = 1 and 1.15, walls with and without the correction) run to t = 0.05 with the ghost-cell
    boundaries of vlbm_set_boundary, the L2 error on u_x beside the printed one, and the time to t.
    value: GLUPS of the 253-cell runs (small lattices of per-node steps: latency-bound)."""
    import torch
    import paper_2607_24059_b300 as vlbm
    import synthetic
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    prec = args.precision if "--precision" in sys.argv else "fp64"
    mu, t_final = 8.0, 0.05
    rows, nodes_253, secs_253 = [], 0, 0.0
    stream = torch.cuda.current_stream()
    launches = 0
    with ClockSampler(local) as clk:
        for n in (75, 112, 168, 253):
            u, phi, dx, nu, u_in = synthetic.poiseuille_channel(n)
            steps = int(math.floor(t_final * mu / dx ** 2 + 1e-6))    # whole steps up to t
            for omega_q in (1.0, 1.15):
                alpha_q = nu / (2.0 * mu * (1.0 / omega_q - 0.5))      # Prop. 1
                for corrected in (False, True):
                    lat = vlbm.Lattice((n, n), dx, nu=0.0, precision=prec, mu=mu, omega_rho=1.2, alpha_rho=0.075,
                                       omega_q=omega_q, alpha_q=alpha_q)
                    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
                    lat.set_channel(u_in, phi_out=0.0, wall_correction=corrected)
                    for k in (64, 16, 4):                                  # first launches, graph capture
                        lat.step(k)
                    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
                    c0 = lat.launch_count()
                    torch.cuda.synchronize()
                    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    start.record(stream)
                    lat.step(steps)
                    end.record(stream)
                    torch.cuda.synchronize()
                    ms = start.elapsed_time(end)
                    launches += lat.launch_count() - c0
                    ux = lat.macros()[1][0].cpu().numpy()
                    lat.close()
                    err = math.sqrt(dx * dx * float(np.sum((ux - u[0]) ** 2)))
                    printed = TABLE2[(n, omega_q, corrected)]
                    rows.append({"cells": n, "omega_q": omega_q, "wall_correction": corrected, "steps": steps,
                                 "l2_error_ux": err, "table2": printed, "ms_to_t": ms})
                    if n == 253:
                        nodes_253 += n * n * steps
                        secs_253 += ms / 1e3
    value = nodes_253 / secs_253 / 1e9
    per_step = secs_253 / (4 * rows[-1]["steps"])
    bpn = 2 * 15 * ELEM_BYTES[prec]
    peak, peak_kind = measured_peaks()
    achieved = bpn * 253 * 253 / per_step / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": rows[-1]["steps"],
        "warmup": 64, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64"}[prec], "data": "synthetic",
        "config": {"workload": "Poiseuille channel of Section 6.2 (Table 2): [0,1]^2, U = 1, Re = 100, mu = 8, "
                               "omega_rho = 6/5, alpha_rho = 3/40, to t = 0.05, ghost-cell boundaries",
                   "storage": prec, "l2": "small lattices (75..253 cells per direction) fit in L2"},
        "table2": rows,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": None, "bytes_per_node": bpn,
                     "kernel": "k_channel_ghosts + k_stream_collide_2d_channel",
                     "note": "253^2 nodes per step: two short launches per step, latency-bound, far from the "
                             "bandwidth roofline by construction"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "poiseuille":
        return run_poiseuille(args)
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "sur256":
        return run_surrogate(args)
    return run_vlbm(args)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Throughput of the fused IB-LBM step (arXiv 2102.01305's method) on one GB300.

Workload (default): the 3D clap-and-fling wing pair - D3Q19, FP32 storage,
256 x 192 x 160 cells, two flat elliptic wings of chord 20 and span 100
(2 x 1576 markers at unit spacing), Re = 100, J = 1e-2, flapping period
4000 steps; every step is the whole hot path (kinematics, interpolation,
implicit solve, spreading, collision + streaming + faces, force reduction).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (the runs share nothing, so there is no collective
on the data path); rank 0 prints one JSON line with the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORLD = int(os.environ.get("WORLD_SIZE", "1"))
RANK = int(os.environ.get("RANK", "0"))
LOCAL_RANK = int(os.environ.get("LOCAL_RANK", "0"))
if WORLD > 1 and "CUDA_VISIBLE_DEVICES" not in os.environ:
    # one GPU per rank; libibl uses the current device of its own runtime (device 0)
    os.environ["CUDA_VISIBLE_DEVICES"] = str(LOCAL_RANK)

METRIC = "IB-LBM D3Q19 GLUPS & % HBM roofline; sweep-serving solves/h, p50/p99 latency"
UNIT = "GLUPS"
FALLBACK_HBM_GBS = 6800.0
# sources the collide-stream kernel is compiled from (lbm.cu up to its
# allocation-free mass section); the recorded DRAM traffic is valid only
# while their hash matches profiles/collide_traffic.txt
COLLIDE_SOURCES = ["paper_2102_01305_gb300/csrc/lbm.cu", "paper_2102_01305_gb300/csrc/lbm_gather.cuh",
                   "paper_2102_01305_gb300/csrc/lattice.cuh"]
LBM_END_MARK = b"// ----------------------------------------------------------------- allocation-free mass"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16dev", "bf16dev", "fp64"])
    ap.add_argument("--workload", default="wings-large", choices=["wings", "wings-large", "tgv"],
                    help="wings-large: the clap-and-fling wing pair at 512x384x320, chord 40 (default, the "
                         "largest single-GPU configuration); wings: the same pair at 256x192x160, chord 20; "
                         "tgv: pure D3Q19 periodic Taylor-Green vortex, u0=0.05, tau=0.6 (roofline sweep)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 256x192x160 wing pair measured after the default workload")
    ap.add_argument("--size", type=int, default=256, help="cube edge of the tgv workload")
    ap.add_argument("--box", default=None,
                    help="NXxNYxNZ: the wing pair of --workload in a box of this size (profiling a smaller case)")
    ap.add_argument("--serving", action="store_true",
                    help="run the serving sweep (Poisson arrivals of clap-and-fling runs) instead")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--mean-gap", type=float, default=2.0, help="mean Poisson inter-arrival gap, s")
    ap.add_argument("--run-steps", type=int, default=10000)
    ap.add_argument("--mix", default="mixed", choices=["mixed", "fp32", "fp16dev", "bf16dev"])
    ap.add_argument("--serve-tune", type=int, default=1, choices=[0, 1],
                    help="serving: 1 per-request launch tuning, 0 library defaults")
    ap.add_argument("--serving-sample", type=int, default=12,
                    help="requests of the short serving sample in the default line (0: none)")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--overlap", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="collide scheduling: -1 automatic, 0 one kernel after the IB chain, 1 split, 2 serial split")
    ap.add_argument("--solver-blocks", type=int, default=0, help="blocks of the implicit solve (0: default)")
    ap.add_argument("--collide-shape", default=None,
                    help="BXxBYxPAIRS: thread block and two-cells-per-thread flag of the one-kernel collide")
    ap.add_argument("--phases", action="store_true", help="also time every phase of the step (events)")
    ap.add_argument("--initial-guess", choices=("extrapolated", "quadratic", "previous", "zero"), default="extrapolated",
                    help="initial guess of each implicit solve")
    ap.add_argument("--refresh-every", type=int, default=0,
                    help="steps between preconditioner rebuilds (0: the library default)")
    ap.add_argument("--ib-sweep", action="store_true",
                    help="IB-stage throughput: interpolate + spread of random point clouds (no solve)")
    ap.add_argument("--ib-markers", default="1000,10000,100000,1000000")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes of the all-cores CPU baseline (0: one per host core)")
    ap.add_argument("--cpu-baseline-worker", default=None)   # internal: run the oracle sample
    return ap.parse_args()


def workload(precision="fp32", scale=1.0, kind="wings", size=256, box=None):
    import workloads as W
    if box:
        # the same wings in another box (profiling): chord and flow as in the workload
        nx, ny, nz = (int(v) for v in box.lower().split("x"))
        if kind == "wings-large":
            return W.clap_fling_3d(nx=nx, ny=ny, nz=nz, chord=40.0, Re=150.0, J=1e-3, period=8000.0,
                                   precision=precision, faces="periodic")
        return W.clap_fling_3d(nx=nx, ny=ny, nz=nz, chord=20.0, precision=precision, faces="periodic")
    if kind == "tgv":
        n = max(8, int(round(size * scale)))
        return W.taylor_green_3d(n=n, u0=0.05, tau=0.6, precision=precision)
    n = lambda v: max(8, int(round(v * scale)))
    # x-periodic box: Zou-He inlet/outlet faces at this tau (0.5126) diverge
    # within a few hundred steps on this 12.8c-long box, on the oracle and the GPU alike
    if kind == "wings-large":
        # 512x384x320 (63M cells), chord 40 (2 x 6283 markers), Re = 150,
        # J = 1e-3, period 8000 steps (tau = 0.5168)
        return W.clap_fling_3d(nx=n(512), ny=n(384), nz=n(320), chord=max(4.0, round(40.0 * scale)),
                               Re=150.0, J=1e-3, period=8000.0 * scale, precision=precision,
                               faces="periodic")
    cfg = W.clap_fling_3d(nx=n(256), ny=n(192), nz=n(160), chord=max(4.0, round(20.0 * scale)),
                          precision=precision, faces="periodic")
    return cfg


def describe(cfg, steps):
    g = cfg["grid"]
    m = [len(b["ds"]) for b in cfg["bodies"]]
    if not m:
        return {"workload": (f"pure D3Q19 periodic Taylor-Green vortex, {g['precision'].upper()}, "
                             f"{g['nx']}^3 cells, u0=0.05, tau=0.6"),
                "cells": g["nx"] * g["ny"] * g["nz"], "markers": 0, "tau": cfg["tau"],
                "steps_timed": steps,
                "l2": ("no flush: populations exceed L2" if g["nx"] ** 3 * 152 > 129e6
                       else "populations fit in L2 (small cube): numbers include L2 reuse")}
    prm = cfg.get("params", {})
    elem = {"fp64": 8, "fp32": 4, "fp16dev": 2, "bf16dev": 2}[g["precision"]]
    buf_mb = g["nx"] * g["ny"] * g["nz"] * 19 * elem / 1e6
    period = 1.0 / prm["f"] if prm.get("f") else float("nan")
    chord = cfg["bodies"][0]["hinge"][0] * 2
    Re = prm["u_tip"] * chord / prm["nu"] if prm.get("nu") else float("nan")
    J = prm["u_inf"] / prm["u_tip"] if prm.get("u_tip") else float("nan")
    return {"workload": (f"3D clap-and-fling wing pair, D3Q19 {g['precision'].upper()}, "
                         f"{g['nx']}x{g['ny']}x{g['nz']} cells, 2 elliptic wings c={cfg['bodies'][0]['hinge'][0]*2:g} "
                         f"span 5c ({m[0]}+{m[1]} markers), Re={Re:.4g}, "
                         f"J={J:.3g} (uniform initial free stream, periodic box), "
                         f"period {period:g} steps"),
            "cells": g["nx"] * g["ny"] * g["nz"], "markers": sum(m), "tau": round(cfg["tau"], 6),
            "steps_timed": steps,
            "l2": f"no flush: every step streams 2 x {buf_mb:.0f} MB of populations, > 129 MB L2"}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]))],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- oracle legs
def oracle_glups(scale: float, steps: int, warm: int = 0, kind: str = "wings", size: int = 256) -> dict:
    """Time the FP64 oracle on a scaled copy of the workload (single thread)."""
    import numpy as np
    from oracle.sim import Simulation
    cfg = workload("fp32", scale, kind, size)
    sim = Simulation(cfg["lattice"], cfg["grid"], cfg["tau"])
    if "u_field" in cfg:
        sim.init_fluid(u=cfg["u_field"])
    else:
        sim.init_fluid(u=np.asarray(cfg["u0"])[:3])
    for b in cfg["bodies"]:
        sim.add_body(b)
    if "reference" in cfg:
        r = cfg["reference"]
        sim.set_reference(r["U_ref"], r["L"], r["rho_ref"])
    sim.step(warm)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    g = cfg["grid"]
    cells = g["nx"] * g["ny"] * g["nz"]
    return {"value": cells * steps / dt / 1e9, "seconds": dt, "steps": steps, "cells": cells,
            "markers": sum(len(b["ds"]) for b in cfg["bodies"]), "box": [g["nx"], g["ny"], g["nz"]]}


def run_oracle_subprocess(scale: float, steps: int, warm: int = 0, timeout: float = 900,
                          kind: str = "wings", size: int = 256) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker",
           f"{scale},{steps},{warm},{kind},{size}"]
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle_parallel(scale: float, steps: int, warm: int, procs: int, timeout: float = 1800,
                        kind: str = "wings", size: int = 256) -> dict:
    """The oracle on every host core: `procs` single-threaded processes each
    step their own copy of the scaled workload at the same time (the oracle
    itself is unchanged and runs one copy per core); aggregate GLUPS = all
    copies' cell updates over the wall time of the slowest."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker",
           f"{scale},{steps},{warm},{kind},{size}"]
    t0 = time.perf_counter()
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
          for _ in range(procs)]
    outs = []
    for pr in ps:
        out, err = pr.communicate(timeout=timeout)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        outs.append(json.loads(out.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    slowest = max(o["seconds"] for o in outs)
    cells = outs[0]["cells"]
    return {"value": procs * cells * steps / slowest / 1e9, "seconds": slowest, "wall": wall, "procs": procs,
            "steps": steps, "cells": cells, "markers": outs[0]["markers"], "box": outs[0]["box"]}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip() + f", {os.cpu_count()} cores"
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ----------------------------------------------------------------------------- replicas
PCG_PHASES = ["stage_z", "spmv_rows", "block_reduce", "barrier1", "alpha", "stage_x", "precond_rows",
              "reduce_barrier2"]


def pcg_trace_summary(tr, iters):
    """Median phase durations (us) of one solve from its timestamps: slots 0-3
    are start / after rebuild / after set-up / end; iteration k (k < 26) has 9
    marks from slot 8 + 9k: scalars ready, then the end of each phase."""
    if not (tr[0] and tr[3]):
        return None
    n = min(iters, 26)
    base = [8 + 9 * k for k in range(n)]
    med = lambda v: round(statistics.median(v), 3) if v else None
    out = {"total_us": (tr[3] - tr[0]) / 1e3, "rebuild_us": (tr[1] - tr[0]) / 1e3,
           "setup_us": (tr[2] - tr[1]) / 1e3}
    if tr[4] and tr[7] and tr[1] - tr[0] > 100000 and tr[4] > tr[0]:
        out["rebuild_first_pivot_us"] = [round((tr[j] - tr[j - 1]) / 1e3, 3) for j in range(5, 8)]
        out["rebuild_first_pivot_us"].insert(0, round((tr[4] - tr[0]) / 1e3, 3))
    prev_end = [tr[2]] + [tr[b + 8] for b in base[:-1]]
    out["scalars_us"] = med([(tr[b] - e) / 1e3 for b, e in zip(base, prev_end)])
    for j, name in enumerate(PCG_PHASES):
        out[name + "_us"] = med([(tr[b + j + 1] - tr[b + j]) / 1e3 for b in base])
    out["iteration_us_median"] = med([(tr[b + 8] - e) / 1e3 for b, e in zip(base, prev_end)])
    if len(tr) > 253 and tr[250] and tr[253] and tr[250] < tr[4] < tr[253]:
        # separable preconditioner: stages A-F of the set-up's first
        # application and stage G with its barrier (block 0's clock)
        marks = [tr[250], tr[4], tr[5], tr[6], tr[7], tr[251], tr[252], tr[253]]
        out["separable_stages_us"] = dict(zip("ABCDEFG", [round((marks[k + 1] - marks[k]) / 1e3, 3)
                                                          for k in range(7)]))
    return out


def aggregate_over_ranks(ms_local: float, cells: int, steps: int, world: int, dist=None, device="cpu"):
    """Whole-job throughput of `world` independent replicas: every rank ran
    `steps` steps of `cells` cells; the job time is the slowest rank's time."""
    ms = ms_local
    if world > 1 and dist is not None:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, cells * steps * world / (ms * 1e-3) / 1e9


# ----------------------------------------------------------------------------- our arm
def traffic_record(collide_hash: str, key: str):
    """DRAM bytes per cell of the collide kernel(s) from one ncu capture
    (profiles/collide_traffic.txt), valid while the collide sources hash the
    same; key "single" (one kernel after the IB chain) or "split"."""
    path = os.path.join(ROOT, "profiles", "collide_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != collide_hash:
        return None
    return rec.get("records", {}).get(key)


def source_hash() -> str:
    h = hashlib.sha256()
    for p in COLLIDE_SOURCES:
        data = open(os.path.join(ROOT, p), "rb").read()
        if p.endswith("lbm.cu") and LBM_END_MARK in data:
            data = data[:data.index(LBM_END_MARK)]
        h.update(data)
    return h.hexdigest()


def measure(ibl, cfg, args, steps, warmup, dist=None, clocks=None, extras=True):
    """Device time of `steps` steps of one workload on the library's stream
    (CUDA events, barrier + synchronize on both sides), after `warmup`
    untimed steps; plus the event-timed collide and IB-chain shares, the
    solver's statistics and, with `extras`, the host enqueue cost and the
    cost of one forced preconditioner rebuild (both after the timed region)."""
    import torch
    ctx = ibl.from_workload(cfg)
    ctx.ibl_set_overlap(args.overlap)
    ctx.ibl_solver_blocks(args.solver_blocks)
    if args.collide_shape:
        bx, by, pairs = (int(v) for v in args.collide_shape.lower().split("x"))
        ctx.ibl_set_collide_shape(bx, by, pairs)
    guess = {"extrapolated": 1, "quadratic": 2, "previous": 0, "zero": -1}[args.initial_guess]
    refresh = args.refresh_every or 384
    if args.refresh_every or args.initial_guess != "extrapolated":
        ctx.ibl_solver_config(refresh, 0.0, guess)
    ctx.ibl_step(warmup)
    ctx.ibl_sync(allow=(ibl.IBL_ENOTCONV,))
    stream = torch.cuda.ExternalStream(ctx.ibl_stream())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ctx.ibl_profile(2 if args.phases else 1)
    l0 = ctx.ibl_launch_count()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    ctx.ibl_step(steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    out = {"ms": ev0.elapsed_time(ev1), "launches": ctx.ibl_launch_count() - l0, "clocks": clk, "status": "ok"}
    try:
        ctx.ibl_sync()
    except ibl.IblError as e:
        out["status"] = str(e)
    bad = (ibl.IBL_ENOTCONV, ibl.IBL_EDIVERGED)
    collide_ms, ib_ms, nprof = ctx.ibl_profile_read()
    out["collide_ms"] = collide_ms / max(nprof, 1)
    out["ib_ms"] = ib_ms / max(nprof, 1)
    out["phases"] = ({k: round(v / max(nprof, 1), 5) for k, v in ctx.ibl_profile_phases().items()}
                     if args.phases else None)
    out["iters"], out["res"], out["refreshes"] = ctx.ibl_solver_stats(allow=bad)
    out["trace"] = None
    if cfg["bodies"]:
        tr = ctx.ibl_solver_trace(allow=bad)
        out["trace"] = pcg_trace_summary(tr, out["iters"]) if len(tr) >= 4 else None
    ok = out["status"] == "ok"
    out["C_L"] = ctx.ibl_forces(0, allow=bad)[0] if ok and cfg["bodies"] else None
    out["host_us"] = out["rebuild_us"] = None
    if ok and extras:
        # host cost of enqueueing a step (the launch queue starts empty, so the
        # calls do not block on the device): compared with the device time per
        # step, it says whether the step is launch-bound
        ctx.ibl_sync(allow=(ibl.IBL_ENOTCONV,))
        ctx.ibl_profile(0)
        t0 = time.perf_counter()
        ctx.ibl_step(16)
        out["host_us"] = round((time.perf_counter() - t0) / 16 * 1e6, 1)
        ctx.ibl_sync(allow=(ibl.IBL_ENOTCONV,))
        if cfg["bodies"]:
            # one more step with a forced preconditioner rebuild: what a
            # rebuild costs at this size (the rebuild interval amortises it)
            t1 = torch.cuda.Event(enable_timing=True)
            t2 = torch.cuda.Event(enable_timing=True)
            ctx.ibl_step(1)
            t1.record(stream)
            ctx.ibl_step(1)
            t2.record(stream)
            t2.synchronize()
            plain = t1.elapsed_time(t2)
            ctx.ibl_solver_config(1, 0.0, guess)
            t1.record(stream)
            ctx.ibl_step(1)
            t2.record(stream)
            t2.synchronize()
            ctx.ibl_sync(allow=(ibl.IBL_ENOTCONV,))
            out["rebuild_us"] = round((t1.elapsed_time(t2) - plain) * 1e3, 1)
            out["refresh_every"] = refresh
    ctx.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2102_01305_gb300 import ibl

    if WORLD > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo",
                                init_method="env://")
    torch.cuda.set_device(0)
    cfg = workload(args.precision, 1.0, args.workload, args.size, args.box)
    g = cfg["grid"]
    cells = g["nx"] * g["ny"] * g["nz"]
    elem = {"fp32": 4, "fp16dev": 2, "bf16dev": 2, "fp64": 8}[args.precision]
    bytes_per_cell = 2 * 19 * elem
    nmark = sum(len(b["ds"]) for b in cfg["bodies"])

    main = measure(ibl, cfg, args, args.steps, args.warmup, dist if WORLD > 1 else None, ClockSampler())
    ms, value = aggregate_over_ranks(main["ms"], cells, args.steps, WORLD, dist if WORLD > 1 else None, "cuda")

    # end to end: host buffers through the public API, copies inside the timed region
    e2e = None
    if RANK == 0 and args.e2e_steps > 0 and cfg["bodies"]:
        e2e = run_e2e(ibl, cfg, args.e2e_steps, cells, warmup=max(args.warmup, 1))

    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak = float(json.load(open(peaks_path))["hbm_gbs"])
        peak_src = "measured"
    else:
        peak, peak_src = FALLBACK_HBM_GBS, "fallback"
    alg_bytes = bytes_per_cell * cells
    achieved = alg_bytes / (main["collide_ms"] * 1e-3) / 1e9
    split = bool(cfg["bodies"]) and (args.overlap == 1 or (args.overlap == -1 and cells >= (1 << 20)
                                                           and nmark <= 8192))
    serial = bool(cfg["bodies"]) and not split and args.overlap == 2
    half_sms = args.overlap == 1 or nmark <= 8192     # the solve's default share of the SMs
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if split:
        pcg_blocks = min(args.solver_blocks or (sms // 2 if half_sms else sms), sms)
        kernel = (f"k_collide_bulk + k_collide_band (split step: the bulk collide runs on the "
                  f"{sms - pcg_blocks} of {sms} SMs the solve leaves free, concurrently with the IB chain)")
        rec_key = "split"
    elif serial:
        kernel = ("k_collide_bulk + k_collide_band (serial split: after the IB chain, the cells outside "
                  "the band on every SM without the band lookup, then the band tiles)")
        rec_key = "split"
    else:
        kernel = "k_collide (collide + stream + faces + IB force, D3Q19, all SMs, after the IB chain)"
        rec_key = "single"
    rec = traffic_record(source_hash(), rec_key) if args.precision == "fp32" and cfg["bodies"] else None
    roofline = {"bound": "hbm", "kernel": kernel,
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": round(rec["traffic_bytes_per_cell"] * cells) if rec else None,
                "traffic_source": rec["source"] if rec else None,
                "algorithmic_bytes_per_launch": alg_bytes,
                "collide_ms_per_step": round(main["collide_ms"], 5),
                "ib_chain_ms_per_step": round(main["ib_ms"], 5),
                "step_ms": round(ms / args.steps, 5),
                "step_frac_of_roofline": round(alg_bytes / (ms / args.steps * 1e-3) / 1e9 / peak, 4)}

    cpu = None
    if RANK == 0 and WORLD == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    secondary = None
    if RANK == 0 and WORLD == 1 and args.workload == "wings-large" and not args.no_secondary:
        cfg1 = workload(args.precision, 1.0, "wings", 256)
        c1 = cfg1["grid"]["nx"] * cfg1["grid"]["ny"] * cfg1["grid"]["nz"]
        r1 = measure(ibl, cfg1, args, max(args.steps, 50), args.warmup, extras=False)
        secondary = {"workload": describe(cfg1, max(args.steps, 50))["workload"],
                     "value": round(c1 * max(args.steps, 50) / (r1["ms"] * 1e-3) / 1e9, 4), "unit": UNIT,
                     "ms_per_step": round(r1["ms"] / max(args.steps, 50), 5),
                     "step_frac_of_roofline": round(bytes_per_cell * c1 / (r1["ms"] / max(args.steps, 50) * 1e-3)
                                                    / 1e9 / peak, 4),
                     "collide_ms_per_step": round(r1["collide_ms"], 5), "ib_chain_ms_per_step": round(r1["ib_ms"], 5),
                     "pcg_iterations_last_step": r1["iters"], "status": r1["status"]}

    ib_sweep = None
    if RANK == 0 and WORLD == 1 and args.workload in ("wings", "wings-large") and not args.no_secondary:
        try:
            ib_sweep = {"grid": "256^3 periodic D3Q19 FP32, Taylor-Green state",
                        "rows": ib_sweep_rows(256, "fp32", [10000, 100000, 1000000], 10, 3),
                        "note": "interpolate (Eq. 17) + spread (Eq. 15) of uniform random points, "
                                "no solve; `bench.py --ib-sweep` for other sizes"}
        except Exception as e:
            ib_sweep = {"error": str(e)[:300]}

    serving = None
    if RANK == 0 and WORLD == 1 and args.serving_sample > 0 and args.workload in ("wings", "wings-large"):
        try:
            serving = run_serving(args.serving_sample, 0.05, 1000, "mixed")
            serving["note"] = ("short sample of the sweep (1000 steps per run, mean gap 0.05 s); "
                               "`bench.py --serving` runs 64 requests x 10000 steps, mean gap 2 s")
        except Exception as e:
            serving = {"error": str(e)[:300]}

    if RANK == 0:
        steps = args.steps
        solver = {"pcg_iterations_last_step": main["iters"], "rel_residual_last_step": main["res"],
                  "preconditioner_rebuilds": main["refreshes"], "trace_last_step": main["trace"],
                  "rebuild_us_forced": main["rebuild_us"]}
        if main["rebuild_us"] is not None:
            # the timed steps hold no scheduled rebuild (the first step builds
            # the preconditioner, the next is due after refresh_every steps)
            solver["ms_per_step_with_rebuilds_amortised"] = round(
                ms / steps + main["rebuild_us"] * 1e-3 / main["refresh_every"], 5)
        line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": WORLD,
                "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms / steps, 5),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp16dev": "f16 storage / f32 compute",
                          "bf16dev": "bf16 storage / f32 compute", "fp64": "f64"}[args.precision],
                "data": "synthetic (seeded workload generator; no dataset)",
                "config": describe(cfg, steps) | {"parallelism": f"replicas x{WORLD}",
                                                  "collide_schedule": {-1: "automatic", 0: "single kernel",
                                                                       1: "split", 2: "serial split"}[args.overlap] +
                                                  (" (split)" if split else (" (serial split)" if serial
                                                                             else " (single kernel)")),
                                                  "solver_blocks": args.solver_blocks or (
                                                      "half the SMs" if half_sms else "all SMs")},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": main["launches"],
                "clocks": main["clocks"], "status": main["status"], "serving_sample": serving, "ib_sweep": ib_sweep,
                "host_enqueue_us_per_step": main["host_us"], "solver": solver,
                "C_L_last_step_body0": main["C_L"]}
        if secondary:
            line["wings_256x192x160"] = secondary
        if main["phases"]:
            line["phase_ms_per_step"] = main["phases"]
        print(json.dumps(line), flush=True)
    if WORLD > 1:
        dist.destroy_process_group()


def cpu_baseline(args) -> dict:
    """The oracle as it stands, timed on this host: one copy per core at
    once (all cores) and one copy alone (single-threaded), each a few steps
    of the workload scaled down so that a copy steps in about a second."""
    scale = 0.25 if args.workload == "wings-large" else 0.5
    procs = args.cpu_procs or os.cpu_count() or 1
    try:
        one = run_oracle_subprocess(scale, 4, 1, kind=args.workload, size=args.size)
        allc = run_oracle_parallel(scale, 4, 1, procs, kind=args.workload, size=args.size)
        box = "x".join(str(v) for v in one["box"])
        return {"value": round(allc["value"], 6), "unit": UNIT, "cores": procs, "kind": "oracle",
                "sample": (f"{procs} copies at once, one per core, each 4 steps (after 1 untimed) of the workload "
                           f"scaled to {box} cells ({one['markers']} markers), numpy FP64, slowest copy "
                           f"{allc['seconds']:.1f} s; host {cpu_model()}"),
                "single_thread": {"value": round(one["value"], 6), "unit": UNIT, "cores": 1,
                                  "sample": f"one copy alone, same sample, {one['seconds']:.1f} s"}}
    except Exception as e:  # the baseline is reported, never required
        return {"value": None, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": f"failed: {e}"[:300]}


def run_e2e(ibl, cfg, steps, cells, warmup=5):
    """Same metric through the public API with host buffers: every step uploads
    both wings' marker positions and wall velocities and reads back the forces.
    `warmup` steps of the same loop run first, untimed, as for the device-timed
    value (the first step builds the solver's preconditioner, and on the
    separable path the span eigenbasis, ~0.3 s once per context)."""
    import numpy as np
    pre = ibl.from_workload(cfg)
    ms = [len(b["ds"]) for b in cfg["bodies"]]
    states = []
    for _ in range(warmup + steps):
        pre.ibl_step(1)
        states.append([pre.ibl_get_markers(b, ms[b], allow=(ibl.IBL_ENOTCONV,))[:2] for b in range(2)])
    pre.close()
    ctx = ibl.from_workload(cfg)

    def one(k):
        for b in range(2):
            X, U = states[k][b]
            ctx.ibl_set_marker_state(b, X, U)
        ctx.ibl_step(1)
        for b in range(2):
            ctx.ibl_forces(b, allow=(ibl.IBL_ENOTCONV,))

    for k in range(warmup):
        one(k)
    ctx.ibl_sync(allow=(ibl.IBL_ENOTCONV,))
    t0 = time.perf_counter()
    for k in range(warmup, warmup + steps):
        one(k)
    dt = time.perf_counter() - t0
    ctx.close()
    h2d = sum(2 * 3 * 8 * m for m in ms)
    d2h = 2 * (3 * 8 + 4)
    return {"value": round(cells * steps / dt / 1e9, 4), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "steps": steps, "warmup": warmup,
            "path": "ibl_set_marker_state (host X, U of both wings) -> ibl_step(1) -> ibl_forces x2"}


# ----------------------------------------------------------------------------- serving
def sweep_requests(n: int, run_steps: int, mix: str, seed: int = 20210203):
    """Requests of the parametric sweep: Re in {75,100,150}, f in {0.05,0.25}
    Hz-equivalent (period 200c or 40c steps), J in {1e-3,1e-2,2}, grid drawn
    uniformly from 96^3, 160x128x112, 256x192x160 with the chord scaled to the
    grid; storage precision FP32 or FP16 deviations 50/50 ("mixed")."""
    import numpy as np
    rng = np.random.default_rng(seed)
    grids = [(96, 96, 96), (160, 128, 112), (256, 192, 160)]
    out = []
    for _ in range(n):
        nx, ny, nz = grids[rng.integers(3)]
        c = float(round(20.0 * nx / 256.0))
        f = [0.05, 0.25][rng.integers(2)]
        prec = mix if mix != "mixed" else ["fp32", "fp16dev"][rng.integers(2)]
        out.append(dict(nx=nx, ny=ny, nz=nz, chord=c, Re=float([75, 100, 150][rng.integers(3)]),
                        period=200.0 * c * 0.05 / f, J=float([1e-3, 1e-2, 2.0][rng.integers(3)]),
                        precision=prec, steps=run_steps))
    return out


def run_serving(n: int, mean_gap: float, run_steps: int, mix: str, budget_frac: float = 0.8, tune: int = 1):
    """Submit a Poisson stream of sweep requests, wait, report solves/h and latency."""
    import numpy as np
    import torch
    from paper_2102_01305_gb300 import ibl
    free, total = torch.cuda.mem_get_info()
    srv = ibl.Server(hbm_budget_bytes=int(free * budget_frac), max_active=16, chunk_steps=50, tune=tune)
    reqs = sweep_requests(n, run_steps, mix)
    rng = np.random.default_rng(7)
    gaps = rng.exponential(mean_gap, size=n)
    t0 = time.perf_counter()
    ids = []
    refused = 0
    admitted = []
    for g, r in zip(gaps, reqs):
        time.sleep(float(g))
        try:
            ids.append(srv.ibl_server_submit(**r))
            admitted.append(r)
        except ibl.IblError as e:
            if e.status != ibl.IBL_EUNSTABLE:
                raise
            refused += 1       # outside the collision's stability range: refused at submission
    srv.ibl_server_wait_all(24 * 3600.0)
    wall = time.perf_counter() - t0
    res = [srv.ibl_server_poll(i) for i in ids]
    load = srv.ibl_server_load()
    srv.close()
    reqs = admitted
    ok = [r for r in res if r["status"] == ibl.IBL_OK]
    lat = sorted(r["finish_s"] - r["submit_s"] for r in ok)
    q = lambda p: float(np.percentile(lat, p)) if lat else None
    cells = sum(rq["nx"] * rq["ny"] * rq["nz"] * rq["steps"] for rq, r in zip(reqs, res) if r["status"] == ibl.IBL_OK)
    return {"solves_per_hour": len(ok) / wall * 3600.0, "requests": n, "completed": len(ok),
            "refused_unstable": refused, "failed": len(res) - len(ok),
            "failure_statuses": sorted({ibl.STATUS_NAMES[r["status"]] for r in res if r["status"] != ibl.IBL_OK}),
            "p50_latency_s": q(50), "p99_latency_s": q(99), "wall_s": wall, "mean_gap_s": mean_gap,
            "steps_per_run": run_steps, "precision_mix": mix, "tune": tune,
            "aggregate_glups": cells / wall / 1e9,
            "scheduler": {"busy_frac": load["busy_s"] / max(load["wall_s"], 1e-9),
                          "enqueue_s": load["enqueue_s"], "build_s": load["build_s"],
                          "retire_s": load["retire_s"], "wall_s": load["wall_s"]},
            "launches": sorted({(r["solve_blocks"], r["overlap"], tuple(r["collide_shape"]))
                                for r in res if r["tuned"]}),
            "runs": [[rq["nx"], rq["chord"], rq["Re"], rq["period"], rq["J"], rq["precision"],
                      ibl.STATUS_NAMES[r["status"]], r["steps_done"]] for rq, r in zip(reqs, res)]}


def ib_sweep_rows(n: int, precision: str, markers, steps: int, warmup: int):
    """Markers/s of the IB stage without the solve: per step one interpolation
    of rho, u* (Eq. 17) and one spreading (Eq. 15) of m random points on an
    n^3 periodic D3Q19 state (a Taylor-Green field after one step), for each
    m of `markers`.  Times are CUDA events around each ABI call on the
    context's stream, so they include the call's launch latency and, for the
    spreading, zeroing and converting the dense 3 x N FP64 output."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2102_01305_gb300 import ibl
    torch.cuda.set_device(0)
    N = n ** 3
    cfg = {"lattice": 19, "tau": 0.6, "grid": W.grid(n, n, n, [W.PERIODIC] * 6, precision=precision),
           "bodies": [], "u_field": W.tgv3d_velocity(n, n, n, 0.05)}
    ctx = ibl.from_workload(cfg)
    del cfg["u_field"]
    ctx.ibl_step(1)
    ctx.ibl_sync()
    stream = torch.cuda.ExternalStream(ctx.ibl_stream())
    dev = dict(dtype=torch.float64, device="cuda")
    out = torch.empty((3, n, n, n), **dev)
    elem = {"fp32": 4, "fp16dev": 2, "bf16dev": 2, "fp64": 8}[precision]
    rows = []
    for m in markers:
        X, V = W.random_markers(m, n, 2.0, n - 2.0, 0.05)
        Xd, Vd, dsd = (torch.as_tensor(a, **dev) for a in (X, V, np.ones(m)))
        U = torch.empty((m, 3), **dev)
        rho = torch.empty(m, **dev)
        ti, ts = [], []
        for k in range(max(warmup, 3) + steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            ctx.ibl_interpolate_points(Xd, U, rho)
            ev[1].record(stream)
            ctx.ibl_spread_points(Xd, Vd, dsd, out)
            ev[2].record(stream)
            ev[2].synchronize()
            if k >= max(warmup, 3):
                ti.append(ev[0].elapsed_time(ev[1]))
                ts.append(ev[1].elapsed_time(ev[2]))
        t_i, t_s = statistics.median(ti), statistics.median(ts)
        union = N * (1.0 - math.exp(-64.0 * m / N))   # cells covered by at least one stencil
        # algorithmic bytes: the interpolation reads 19 populations on the
        # covered cells and 36 B of point data; the spreading writes 24 B
        # (3 x FP64) on the covered cells and reads 64 B of point data
        b_i = union * 19 * elem + m * 24 + m * 32
        b_s = union * 24 + m * 64
        rows.append({"markers": m, "interpolate_ms": round(t_i, 4), "spread_ms": round(t_s, 4),
                     "markers_per_s": m / ((t_i + t_s) * 1e-3),
                     "covered_cells_frac": round(union / N, 4),
                     "interpolate_GBs": round(b_i / (t_i * 1e-3) / 1e9, 1),
                     "spread_GBs": round(b_s / (t_s * 1e-3) / 1e9, 1)})
        del Xd, Vd, dsd, U, rho
    ctx.close()
    return rows


def run_ib_sweep(args):
    """The IB-stage sweep of ib_sweep_rows as its own JSON line."""
    clocks = ClockSampler()
    clocks.start()
    rows = ib_sweep_rows(args.size, args.precision, [int(v) for v in args.ib_markers.split(",")],
                         args.steps, args.warmup)
    clk = clocks.stop()
    best = max(rows, key=lambda r: r["markers_per_s"])
    print(json.dumps({"metric": "IB-stage markers/s (interpolate + spread, no solve)",
                      "value": round(best["markers_per_s"], 1), "unit": "markers/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": max(args.warmup, 3), "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
                      "data": "synthetic (uniform random points in [2, n-2)^3, velocities in [-0.05, 0.05]^3)",
                      "config": {"workload": f"IB sweep on a {args.size}^3 periodic D3Q19 grid",
                                 "l2": "no flush: the populations (2 x 19 x N) exceed L2",
                                 "timing": "CUDA events around each ABI call (median)"},
                      "sweep": rows, "clocks": clk}), flush=True)


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    if WORLD > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
        if RANK != 0:
            dist.destroy_process_group()
            return
    # the oracle as it stands, one copy per host core at once; each copy's
    # step is one oracle step of the workload scaled so that the whole
    # warm-up + timed run takes about two minutes
    budget = 120.0
    per_step = budget / max(1, args.steps + args.warmup)
    cells_target = max(6000.0, min(1.0e6, per_step * 2.0e5))
    full = args.size ** 3 if args.workload == "tgv" else (512 * 384 * 320 if args.workload == "wings-large"
                                                          else 256 * 192 * 160)
    scale = (cells_target / full) ** (1.0 / 3.0)
    procs = args.cpu_procs or os.cpu_count() or 1
    r = run_oracle_parallel(scale, args.steps, args.warmup, procs, timeout=3600, kind=args.workload,
                            size=args.size)
    cfg = workload("fp32", 1.0, args.workload, args.size)
    box = f"{r['box'][0]}x{r['box'][1]}x{r['box'][2]}"
    line = {"impl": "reference", "metric": METRIC, "value": round(r["value"], 6), "unit": UNIT,
            "n_gpus": WORLD, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(r["seconds"] / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(cfg, args.steps) | {"parallelism": "oracle, rank 0 only"},
            "cpu_baseline": {"value": round(r["value"], 6), "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": (f"{procs} copies at once, one per core, each step one oracle step of the "
                                        f"workload scaled to {box} cells ({r['markers']} markers); numpy FP64; "
                                        f"host {cpu_model()}")},
            "e2e": {"value": round(r["value"], 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if WORLD > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.cpu_baseline_worker:
        scale, steps, warm, kind, size = args.cpu_baseline_worker.split(",")
        print(json.dumps(oracle_glups(float(scale), int(steps), int(warm), kind, int(size))))
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.ib_sweep:
        run_ib_sweep(args)
    elif args.serving:
        r = run_serving(args.requests, args.mean_gap, args.run_steps, args.mix, tune=args.serve_tune)
        print(json.dumps({"metric": METRIC, "value": round(r["solves_per_hour"], 2), "unit": "solves/h",
                          "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "data": "synthetic (seeded sweep of the paper's Re, f, J grid)",
                          "config": {"workload": "serving sweep of clap-and-fling runs",
                                     "parallelism": "continuous batching, one stream per run"},
                          "serving": r}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

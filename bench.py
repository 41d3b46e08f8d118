"""Benchmark: GKTL-batched ensemble D2Q9 stepping on one GB300.

Workload (one "step" = one GKTL cloning period, the whole hot path once):
64 clones of a 1024 x 256 periodic channel, 32 x 32 square obstacle at
x = 256, tau = 0.505, body force g_x = 1e-6, FP32 populations; per period
500 fused stream-collide steps with drag, the window integral of the drag,
GKTL weights and resampling with k*sigma = 1, and cloning with the App. D
perturbation (eps = 0.002, 10 snapshots).  Metric: GLUPS (lattice-site
updates per second over all sites), plus the fused step's HBM roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain FP64, one thread per process)
on a bounded sample of the same workload.  Under torchrun every rank runs an
independent ensemble (replicas, weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PERIOD = 500
TAU, GX = 0.505, 1e-6
# the synthetic workloads: channel nx x ny, clones, obstacle side at x = nx/4,
# and whether a step includes GKTL cloning (the default is the GKTL workload)
WORKLOADS = {
    "gktl": dict(nx=1024, ny=256, clones=64, side=32, cloning=True,
                 name="GKTL batched ensemble: N={n} clones, D2Q9 LBGK {st}, 1024x256, 32x32 obstacle at x=256, "
                      "tau=0.505, g_x=1e-06, resample every 500 steps"),
    "precision": dict(nx=2048, ny=512, clones=16, side=64, cloning=False,
                      name="Precision sweep: N={n} clones, 2048x512, 64x64 obstacle at x=512, tau=0.505, g_x=1e-06, "
                           "populations stored as {st}, 500 steps per step"),
    "ams": dict(nx=512, ny=128, clones=256, side=16, cloning=False,
                name="AMS initial ensemble: N={n} trajectories, 512x128, 16x16 obstacle at x=128, tau=0.505, "
                     "g_x=1e-06, {st}, 500 steps per step"),
}


def workload(args):
    w = dict(WORKLOADS[args.workload])
    w["clones"] = args.clones or w["clones"]
    nx, ny, side = w["nx"], w["ny"], w["side"]
    w["obst"] = (nx // 4 - side // 2, ny // 2 - side // 2, side, side)
    return w
EPS, N_SNAP = 0.002, 10
K_SIGMA = 1.0
SIGMA_DRAG = 1e-3        # drag scale used to set k (k = K_SIGMA / (SIGMA_DRAG * PERIOD))
BYTES_PER_SITE = 72      # FP32: 9 loads + 9 stores of 4 bytes
METRIC = "Ensemble D2Q9 GLUPS & HBM-roofline fraction; time-to-return-time vs plain"
# DRAM traffic of one fused-step launch measured by ncu on this workload, and
# the kernel source it was measured on (reported only while the source matches)
NCU_TRAFFIC = {"sha": "12cee4d507c8406e", "bytes_per_site": 68.5474}  # mean of 3 launches, 64 clones


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("lbm_step.cuh", "lbm_device.cuh", "step_fp32.cu"):
        with open(os.path.join(ROOT, "paper_2005_09323_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, index: int):
        self.proc = None
        self.index = index
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 6:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx = float(parts[1])
                except ValueError:
                    continue
                for n, v in zip(names, parts[2:]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def _oracle_worker(args):
    steps, seed, barrier, nx, ny, obst = args
    sys.path.insert(0, ROOT)
    import oracle
    c = oracle.cfg(nx, ny, obstacle=obst, tau=TAU, gx=GX)
    f = oracle.init(c, seed, 0, 0.01)
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    oracle.run(c, f, steps)
    return time.perf_counter() - t0


def oracle_rate(steps_per_proc: int, procs: int, w):
    """Aggregate oracle GLUPS over `procs` single-threaded processes (spawned),
    each advancing one clone of the workload's channel by steps_per_proc steps."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    geo = (w["nx"], w["ny"], w["obst"])
    if procs == 1:
        dt = _oracle_worker((steps_per_proc, 0, None) + geo)
        times = [dt]
    else:
        with ctx.Manager() as m:
            barrier = m.Barrier(procs)
            with ctx.Pool(procs) as pool:
                times = pool.map(_oracle_worker, [(steps_per_proc, s, barrier) + geo for s in range(procs)])
    updates = w["nx"] * w["ny"] * steps_per_proc * procs
    wall = max(times)
    return updates / wall / 1e9, wall, sum(times)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = cpu_cores()
    w = workload(args)
    steps_per_proc = max(1, int(20 * 1024 * 256 / (w["nx"] * w["ny"])))
    vals, walls = [], []
    for _ in range(args.warmup):
        oracle_rate(1, 1, w)
    for _ in range(args.steps):
        v, wall, _ = oracle_rate(steps_per_proc, cores, w)
        vals.append(v)
        walls.append(wall)
    value = statistics.median(vals)
    sample = (f"{cores} processes x 1 clone of {w['nx']}x{w['ny']} x {steps_per_proc} steps per step "
              f"(of {w['clones']} clones x {PERIOD} steps per workload step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def workload_config(args):
    w = workload(args)
    st = {"fp32": "FP32", "fp16": "shifted FP16", "bf16": "shifted BF16"}[args.storage]
    state_gb = 2 * w["clones"] * 9 * w["nx"] * w["ny"] * (4 if args.storage == "fp32" else 2) / 1e9
    cfg = {"workload": w["name"].format(n=w["clones"], st=st), "clones": w["clones"], "grid": [w["nx"], w["ny"]],
           "steps_per_step": PERIOD, "storage": args.storage,
           "l2": f"working set {state_gb:.2f} GB of populations (two buffers, >> 129 MB L2); no flush needed",
           "parallelism": f"replicas x{args.gpus}"}
    if w["cloning"]:
        cfg.update({"k_sigma": K_SIGMA, "eps": EPS, "n_snapshots": N_SNAP})
    return cfg


# ---------------------------------------------------------------- GPU
def run_ours(args):
    import numpy as np
    import torch

    from paper_2005_09323_gb300 import build
    from paper_2005_09323_gb300 import lbmrare as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if not os.path.exists(build.LIB):
        raise RuntimeError("liblbmrare.so missing: run __graft_entry__.build() first")
    L.lib()

    # CPU baseline first (spawned processes, before the GPU is touched)
    w = workload(args)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = cpu_cores()
        spp = max(1, int(20 * 1024 * 256 / (w["nx"] * w["ny"])))
        v, wall, cpu_s = oracle_rate(spp, cores, w)
        cpu = {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{cores} single-threaded oracle processes, each one clone of {w['nx']}x{w['ny']} for "
                         f"{spp} steps ({cpu_s:.1f} s of CPU work, {wall:.1f} s wall)"}

    stream = torch.cuda.current_stream()
    total_periods = args.warmup + args.steps + 2 * (args.warmup + args.steps) + 2
    nx, ny = w["nx"], w["ny"]
    cfg = L.config(nx, ny, obstacle=w["obst"], tau=TAU, gx=GX, max_steps=PERIOD * total_periods,
                   n_snapshots=N_SNAP, init_amp=0.01, storage=args.storage)
    n_clones = w["clones"]
    e = L.lbm_ensemble_create(cfg, n_clones, 1000 + rank, stream)
    if args.variant == "auto":
        variant = L.lbm_ensemble_autotune(e)
    else:
        variant = int(args.variant)
        L.lbm_ensemble_set_variant(e, variant)
    vinfo = L.lbm_step_variant_info(variant)
    k = K_SIGMA / (SIGMA_DRAG * PERIOD)
    s = torch.zeros(n_clones, dtype=torch.float64, device="cuda")
    W = torch.zeros_like(s)
    logR = torch.zeros(1, dtype=torch.float64, device="cuda")
    parent = torch.zeros(n_clones, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    state = {"t": 0, "it": 0}

    def gktl_period():
        t0 = state["t"]
        L.lbm_ensemble_step(e, PERIOD)
        L.lbm_ensemble_window_sum(e, t0, t0 + PERIOD, k, s)
        if w["cloning"]:
            L.gktl_weights(s, W, logR, stream)
            L.gktl_select(W, 7, state["it"], parent, status, stream)
            L.lbm_ensemble_clone(e, parent, EPS, 7, state["it"])
        state["t"] += PERIOD
        state["it"] += 1

    # snapshot bank from the initial ensemble (App. D: arbitrary flow states)
    L.lbm_ensemble_step(e, PERIOD)
    state["t"] += PERIOD
    L.lbm_ensemble_set_snapshots(e, list(range(N_SNAP)))
    for _ in range(args.warmup):
        gktl_period()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    L.lbm_ensemble_set_timing(e, True)
    L.lbm_ensemble_kernel_time(e, reset=True)
    launches0 = L.lbm_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            gktl_period()
        ev1.record(stream)
        barrier()
    launches = L.lbm_launch_count() - launches0
    st_ms, st_launches = L.lbm_ensemble_kernel_time(e, reset=True)
    L.lbm_ensemble_set_timing(e, False)
    ms = ev0.elapsed_time(ev1)
    if status.item() != 0:
        raise RuntimeError(f"gktl_select status {status.item()}")

    # end to end through the C ABI with host buffers: the drag series goes to
    # the host, the GKTL exponents are formed there and sent back, the parents
    # come back to the host
    pinned_s = torch.zeros(n_clones, dtype=torch.float64).pin_memory()
    pinned_p = torch.zeros(n_clones, dtype=torch.int32).pin_memory()
    drag_host = np.zeros((n_clones, PERIOD))
    e2e_steps = max(1, args.steps // 2)

    def e2e_period():
        t0 = state["t"]
        L.lbm_ensemble_step(e, PERIOD)
        L.lbm_ensemble_drag(e, t0, t0 + PERIOD, drag_host)       # D2H, waits
        pinned_s.numpy()[:] = k * drag_host.sum(axis=1)
        s.copy_(pinned_s, non_blocking=True)                      # H2D
        if w["cloning"]:
            L.gktl_weights(s, W, logR, stream)
            L.gktl_select(W, 7, state["it"], parent, status, stream)
            pinned_p.copy_(parent, non_blocking=True)             # D2H
            L.lbm_ensemble_clone(e, parent, EPS, 7, state["it"])
        torch.cuda.current_stream().synchronize()
        state["t"] += PERIOD
        state["it"] += 1

    e2e_period()
    barrier()
    t_e2e = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_period()
    barrier()
    e2e_s = time.perf_counter() - t_e2e

    L.lbm_ensemble_destroy(e)

    if dist is not None:
        tt = torch.tensor([ms, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms, e2e_s = tt.tolist()
    sites = n_clones * nx * ny
    updates = sites * PERIOD * args.steps * world
    value = updates / (ms / 1e3) / 1e9
    e2e_value = sites * PERIOD * e2e_steps * world / e2e_s / 1e9
    hbm, peak_kind = peaks()
    avg_launch_ms = st_ms / max(st_launches, 1)
    bytes_per_site = BYTES_PER_SITE if args.storage == "fp32" else BYTES_PER_SITE // 2
    achieved = bytes_per_site * sites / (avg_launch_ms / 1e3) / 1e9
    traffic = None
    if (NCU_TRAFFIC["sha"] == kernel_sha() and NCU_TRAFFIC["bytes_per_site"] and args.workload == "gktl"
            and args.storage == "fp32"):
        traffic = NCU_TRAFFIC["bytes_per_site"] * sites
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": f"step_kernel<{args.storage}, vec={vinfo[1]}, warps={vinfo[2]}>",
                         "peak_kind": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_site": bytes_per_site,
                         "avg_launch_us": avg_launch_ms * 1e3},
            "e2e": {"value": e2e_value, "unit": "GLUPS", "h2d_bytes_per_step": 8 * n_clones,
                    "d2h_bytes_per_step": 8 * n_clones * PERIOD + 4 * n_clones},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--variant", default="auto",
                    help="fused-step variant index, or 'auto' to autotune (profiling captures fix it)")
    ap.add_argument("--clones", type=int, default=0,
                    help="ensemble size (default: the workload's; smaller only for profiling captures)")
    ap.add_argument("--workload", default="gktl", choices=sorted(WORKLOADS))
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

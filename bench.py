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
import re
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
    "direct": dict(nx=1024, ny=256, clones=64, side=32, cloning=False,
                   name="Direct sampling (Sec. 3): N={n} independent trajectories, D2Q9 LBGK {st}, 1024x256, "
                        "32x32 obstacle at x=256, tau=0.505, g_x=1e-06, 500 steps per step; drag autocorrelation "
                        "and waiting-time return times over the run"),
    "open": dict(nx=513, ny=129, clones=64, side=16, cloning=False, open=True,
                 name="Open channel of Sec. 2: N={n} independent trajectories, D2Q9 {st}, 513x129, 16x16 square at "
                      "the centre, entrance grid of 8-row bars every 16 rows at x=16..23, parabolic inlet u_c=0.05, "
                      "regularized outlet, sponge of 128 columns up to tau=1, tau=0.501 (Re_grid=1200), 500 steps "
                      "per step; drag autocorrelation and waiting-time return times over the run"),
}
# open channel of Sec. 2: Re_grid = u_c (R/2) / nu = 1200 with u_c = 0.05, R = 16
OPEN_UC = 0.05
OPEN_TAU = 0.5 + 3.0 * OPEN_UC * 8 / 1200
OPEN_GRID = (16, 8, 8, 8)     # x0, width, bar rows, gap rows
OPEN_SPONGE = (128, 1.0)      # columns, tau at the outlet


def workload(args):
    w = dict(WORKLOADS[args.workload])
    w["clones"] = args.clones or w["clones"]
    nx, ny, side = w["nx"], w["ny"], w["side"]
    if w.get("open"):  # the square at the centre of the channel
        w["obst"] = (nx // 2 - side // 2, ny // 2 - side // 2, side, side)
    else:
        w["obst"] = (nx // 4 - side // 2, ny // 2 - side // 2, side, side)
    coll = getattr(args, "collision", None)
    w["collision"] = coll or ("cm" if w.get("open") else "bgk")
    return w


def channel_kwargs(w) -> dict:
    """geometry and flow of the workload's channel, in the keywords that the
    library's config() and the oracle's cfg() share"""
    if w.get("open"):
        return dict(tau=OPEN_TAU, gx=0.0, open_x=1, u_in=OPEN_UC, grid=OPEN_GRID, sponge_len=OPEN_SPONGE[0],
                    sponge_tau=OPEN_SPONGE[1])
    return dict(tau=TAU, gx=GX)
EPS, N_SNAP = 0.002, 10
CHECK_STEPS, CHECK_PERIOD = 5000, 1000  # perturbation check: steps per bench step, perturbation period (tau_c / 2)
K_SIGMA = 1.0
SIGMA_DRAG = 1e-3        # drag scale used to set k (k = K_SIGMA / (SIGMA_DRAG * PERIOD))
BYTES_PER_SITE = 72      # FP32: 9 loads + 9 stores of 4 bytes
METRIC = "Ensemble D2Q9 GLUPS & HBM-roofline fraction; time-to-return-time vs plain"
# DRAM traffic of one fused-step launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of launches of the full workload), per site,
# with the kernel sources it was measured on: reported only while they match
NCU_TRAFFIC = {
    ("gktl", "step_kernel<fp32, vec=4>"): {
        "files": ("lbm_step.cuh", "lbm_device.cuh", "step_params.h", "step_fp32.cu"),
        "sha": "241df406e4de695e", "bytes_per_site": 68.4597},
    ("precision", "step_rows_kernel<fp16, vec=4>"): {
        "files": ("lbm_step_rows.cuh", "async_copy.cuh", "lbm_step.cuh", "lbm_device.cuh", "step_params.h",
                  "step_fp16.cu"),
        "sha": "9c24a2e7bd8f6b3e", "bytes_per_site": 32.5115},
    # both kernels of an open-channel step (the step kernel and the outlet kernel)
    ("open", "step_kernel<fp32, vec=4, open> + open_bc_kernel"): {
        "files": ("lbm_step.cuh", "lbm_device.cuh", "step_params.h", "step_open_fp32.cu"),
        "sha": "3f91ba9496814b0e", "bytes_per_site": 59.1880},
}


def traffic_key(label: str) -> str:
    """a kernel label without its warps per block, which leave the DRAM
    traffic of a launch unchanged (the loads depend on the vector width)"""
    return re.sub(r", warps=\d+", "", label)


def kernel_sha(files=NCU_TRAFFIC[("gktl", "step_kernel<fp32, vec=4>")]["files"]) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2005_09323_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_label(L, variant: int, storage: str) -> str:
    _, vec, warps = L.lbm_step_variant_info(variant)
    name = "step_rows_kernel" if L.lbm_step_variant_kind(variant) == 1 else "step_kernel"
    return f"{name}<{storage}, vec={vec}, warps={warps}>"


def max_over_ranks(dist, values, device="cpu"):
    """Each rank's timings -> their maxima over all ranks (the slowest rank
    sets the job's time).  dist = None: a single process."""
    import torch
    if dist is None:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_glups(sites_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the lattice-site updates of all ranks over the
    job's time (replicas: every rank advances its own ensemble)."""
    return sites_per_rank * steps * world / seconds / 1e9


def replica_seed(rank: int) -> int:
    """Each rank's ensemble is an independent replica with its own seed."""
    return 1000 + rank


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi clock and throttle-reason samples every 200 ms while the
    timed region runs, kept as CSV in $LBM_CLOCKS_DIR (default: the system's
    temporary directory)"""

    def __init__(self, index: int):
        import tempfile
        self.proc = None
        self.index = index
        out = os.environ.get("LBM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_{os.getpid()}.csv")

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
    steps, seed, barrier, nx, ny, obst, collision, chan = args
    sys.path.insert(0, ROOT)
    import oracle
    c = oracle.cfg(nx, ny, obstacle=obst, collision=1 if collision == "cm" else 0, **chan)
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
    geo = (w["nx"], w["ny"], w["obst"], w.get("collision", "bgk"), channel_kwargs(w))
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


def cpu_baseline(w, cores: int) -> dict:
    """the oracle as it stands, timed on `cores` host cores over a bounded
    sample of the workload (each process one clone, about 20 steps of a
    1024 x 256 lattice's worth of sites): aggregate and single-process rates"""
    spp = max(1, int(20 * 1024 * 256 / (w["nx"] * w["ny"])))
    v, wall, cpu_s = oracle_rate(spp, cores, w)
    return {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle", "per_core": v * wall / cpu_s,
            "sample": f"{cores} single-threaded oracle processes, each one clone of {w['nx']}x{w['ny']} for "
                      f"{spp} steps ({cpu_s:.1f} s of CPU work, {wall:.1f} s wall)"}


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
    vals, walls, per_core = [], [], []
    for _ in range(args.warmup):
        oracle_rate(1, 1, w)
    for _ in range(args.steps):
        v, wall, cpu_s = oracle_rate(steps_per_proc, cores, w)
        vals.append(v)
        walls.append(wall)
        per_core.append(v * wall / cpu_s)  # one process: updates per second of its own time
    value = statistics.median(vals)
    sample = (f"{cores} processes x 1 clone of {w['nx']}x{w['ny']} x {steps_per_proc} steps per step "
              f"(of {w['clones']} clones x {PERIOD} steps per workload step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": sample,
                         "per_core": statistics.median(per_core)},
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
    if w["collision"] == "cm":
        cfg["workload"] += ", central-moment collision (shear 1/tau, bulk/3rd/4th-order rates 1)"
        cfg["collision"] = "central moments"
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
        cpu = cpu_baseline(w, cpu_cores())

    stream = torch.cuda.current_stream()
    total_periods = args.warmup + args.steps + 2 * (args.warmup + args.steps) + 2
    nx, ny = w["nx"], w["ny"]
    cfg = L.config(nx, ny, obstacle=w["obst"], max_steps=PERIOD * total_periods, n_snapshots=N_SNAP, init_amp=0.01,
                   storage=args.storage, collision=w["collision"], **channel_kwargs(w))
    n_clones = w["clones"]
    e = L.lbm_ensemble_create(cfg, n_clones, replica_seed(rank), stream)
    if args.variant == "auto":
        variant = L.lbm_ensemble_autotune(e)
    else:
        variant = int(args.variant)
        L.lbm_ensemble_set_variant(e, variant)
    label = kernel_label(L, variant, args.storage)
    if w.get("open"):  # the open instantiation, with the outlet kernel in each timed step
        label = label[:-1] + ", open> + open_bc_kernel"
    k = K_SIGMA / (SIGMA_DRAG * PERIOD)
    s = torch.zeros(n_clones, dtype=torch.float64, device="cuda")
    W = torch.zeros_like(s)
    logR = torch.zeros(1, dtype=torch.float64, device="cuda")
    parent = torch.zeros(n_clones, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    state = {"t": 0, "it": 0}
    bank = [i * n_clones // N_SNAP for i in range(N_SNAP)]

    def gktl_period():
        t0 = state["t"]
        L.lbm_ensemble_step(e, PERIOD)
        L.lbm_ensemble_window_sum(e, t0, t0 + PERIOD, k, s)
        if w["cloning"]:
            L.gktl_weights(s, W, logR, stream)
            L.gktl_select(W, 7, state["it"], parent, status, stream)
            L.lbm_ensemble_set_snapshots(e, bank)  # contemporaneous App. D directions
            L.lbm_ensemble_clone(e, parent, EPS, 7, state["it"])
        state["t"] += PERIOD
        state["it"] += 1

    # snapshot bank from the initial ensemble (App. D: arbitrary flow states)
    L.lbm_ensemble_step(e, PERIOD)
    state["t"] += PERIOD
    L.lbm_ensemble_set_snapshots(e, bank)
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
            L.lbm_ensemble_set_snapshots(e, bank)
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

    direct = None
    if args.workload in ("direct", "open"):  # statistics of the run after the first period (Sec. 3)
        t0s, t1s = PERIOD, state["t"]
        lag = min(2000, t1s - t0s - 1)
        cdev = torch.zeros(lag + 1, dtype=torch.float64, device="cuda")
        tau_c = L.lbm_drag_autocorrelation(e, t0s, t1s, lag, cdev)
        dh = np.zeros((n_clones, t1s - t0s))
        L.lbm_ensemble_drag(e, t0s, t1s, dh)
        mu, sd = float(dh.mean()), float(dh.std())
        zs = [1.0, 2.0, 3.0]
        lv = torch.tensor([mu + z * sd for z in zs], dtype=torch.float64, device="cuda")
        gap = max(tau_c, 1)
        ev, rt = L.lbm_drag_return_times(e, t0s, t1s, lv, gap)
        direct = {"steps": [t0s, t1s], "drag_mean": mu, "drag_std": sd, "tau_c_steps": tau_c,
                  "return_times": [{"level": f"mean + {z:g} std", "events": int(n_ev),
                                    "r_steps": (None if not np.isfinite(r) else float(r))}
                                   for z, n_ev, r in zip(zs, ev, rt)],
                  "note": ("flow developing from the inlet profile over the run: not yet stationary"
                           if w.get("open") else "flow accelerating from rest under g_x: not stationary over the run")}

    L.lbm_ensemble_destroy(e)

    ms, e2e_s = max_over_ranks(dist, [ms, e2e_s], device="cuda")
    sites = n_clones * nx * ny
    value = job_glups(sites, PERIOD * args.steps, world, ms / 1e3)
    e2e_value = job_glups(sites, PERIOD * e2e_steps, world, e2e_s)
    hbm, peak_kind = peaks()
    avg_launch_ms = st_ms / max(st_launches, 1)
    bytes_per_site = BYTES_PER_SITE if args.storage == "fp32" else BYTES_PER_SITE // 2
    achieved = bytes_per_site * sites / (avg_launch_ms / 1e3) / 1e9
    traffic = None
    rec = NCU_TRAFFIC.get((args.workload, traffic_key(label)))
    if rec and rec["sha"] == kernel_sha(rec["files"]) and not args.clones:
        traffic = rec["bytes_per_site"] * sites
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": label,
                         "peak_kind": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_site": bytes_per_site,
                         "avg_launch_us": avg_launch_ms * 1e3},
            "e2e": {"value": e2e_value, "unit": "GLUPS", "h2d_bytes_per_step": 8 * n_clones,
                    "d2h_bytes_per_step": 8 * n_clones * PERIOD + 4 * n_clones},
            "gpu_launches": launches,
            "clocks": clocks,
            # GLUPS over fluid sites only (the solid cells are updated too)
            "fluid_only": {"value": value * (1.0 - solid_cells(w) / (nx * ny)), "unit": "GLUPS",
                           "fluid_fraction": 1.0 - solid_cells(w) / (nx * ny)},
        }
        if direct is not None:
            line["direct_sampling"] = direct
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- precision report
def run_precision_report(args):
    """Reduced-precision storage against FP32 (and FP32 against the FP64
    oracle): the precision sweep, 16 clones of 2048 x 512 with a 64 x 64
    obstacle, tau = 0.505, g_x = 1e-6, 5000 steps from identical seeded states."""
    import numpy as np
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    w = WORKLOADS["precision"]
    nx, ny, n = w["nx"], w["ny"], w["clones"]
    obst = (nx // 4 - w["side"] // 2, ny // 2 - w["side"] // 2, w["side"], w["side"])
    T = max(200, args.steps)
    stream = torch.cuda.current_stream()
    series, mass = {}, {}
    storages = ["fp32", "fp16", "bf16"] + [s_ for s_ in ("fp16_sr", "bf16_sr") if s_ in L.STORAGE_NAMES]
    for st in storages:
        cfg = L.config(nx, ny, obstacle=obst, tau=TAU, gx=GX, max_steps=T, storage=st)
        e = L.lbm_ensemble_create(cfg, n, 21, stream)
        m0, _, _ = L.lbm_ensemble_moments(e, n)
        L.lbm_ensemble_step(e, T)
        d = np.zeros((n, T))
        L.lbm_ensemble_drag(e, 0, T, d)
        m1, _, _ = L.lbm_ensemble_moments(e, n)
        series[st], mass[st] = d, float(np.max(np.abs(m1 - m0) / m0))
        L.lbm_ensemble_destroy(e)
    # FP32 against the FP64 oracle, one clone, first 100 steps
    import oracle
    oc = oracle.cfg(nx, ny, obstacle=obst, tau=TAU, gx=GX)
    cfg = L.config(nx, ny, obstacle=obst, tau=TAU, gx=GX, max_steps=100)
    e = L.lbm_ensemble_create(cfg, 1, 21, stream)
    L.lbm_ensemble_step(e, 100)
    d32 = np.zeros((1, 100))
    L.lbm_ensemble_drag(e, 0, 100, d32)
    f32 = L.lbm_ensemble_get_populations(e, 0, nx, ny)
    L.lbm_ensemble_destroy(e)
    f64, d64 = oracle.run(oc, oracle.init(oc, 21, 0, 0.01), 100)
    ref = series["fp32"]
    half = T // 2
    report = {"fp32_vs_fp64_oracle_100_steps": {
        "population_rel_err": float(np.abs(f32 - f64).max() / np.abs(f64).max()),
        "drag_rel_err": float(np.abs(d32[0] - d64).max() / np.abs(d64).max())}}

    def ks(a, b):
        a, b = np.sort(a), np.sort(b)
        grid = np.concatenate([a, b])
        return float(np.max(np.abs(np.searchsorted(a, grid, side="right") / len(a)
                                   - np.searchsorted(b, grid, side="right") / len(b))))
    for st, d in series.items():
        tail, rtail = d[:, half:].ravel(), ref[:, half:].ravel()
        report[st] = {
            "drag_series_rel_err_vs_fp32": float(np.abs(d - ref).max() / np.abs(ref).max()),
            "drag_series_rel_err_first_200": float(np.abs(d[:, :200] - ref[:, :200]).max()
                                                   / np.abs(ref[:, :200]).max()),
            "mass_drift": mass[st],
            "drag_mean_rel_dev": float((tail.mean() - rtail.mean()) / abs(rtail.mean())),
            "drag_std_rel_dev": float((tail.std() - rtail.std()) / rtail.std()),
            "drag_ks_vs_fp32": ks(tail, rtail),
            "drag_mean_second_half": float(tail.mean()), "drag_std_second_half": float(tail.std())}
    print(json.dumps({"metric": "reduced-precision storage error report", "steps": T,
                      "config": {"workload": f"Precision sweep: N={n} clones, {nx}x{ny}, {w['side']}x{w['side']} "
                                             f"obstacle, tau={TAU}, g_x={GX}, {T} steps"},
                      "report": report}))


# chaotic small open channel of the long-run comparisons: 129 x 33, square of
# side 8 at the centre, bars of 4 rows every 8 from x = 8, 32-column sponge to
# tau = 1, central moments, tau = 0.5015, u_c = 0.08 (drag correlation time
# about 340 steps; a 1e-6 change of one population grows to the drag's
# fluctuation size within about 4000 steps)
CHAOTIC = dict(nx=129, ny=33, obstacle=(60, 12, 8, 8), tau=0.5015, open_x=1, u_in=0.08, grid=(8, 4, 4, 4),
               sponge_len=32, sponge_tau=1.0)


def _chaotic_oracle_drag(job):
    """one oracle trajectory of the chaotic channel: (seed, clone, steps) -> drag"""
    import oracle
    seed, clone, steps = job
    kw = dict(CHAOTIC)
    c = oracle.cfg(kw.pop("nx"), kw.pop("ny"), obstacle=kw.pop("obstacle"), collision=1, **kw)
    return oracle.run(c, oracle.init(c, seed, clone, 0.01), steps)[1]


def run_long_run_precision(args):
    """Long-run drag statistics past the predictability horizon in the chaotic
    small open channel: shifted FP16 and BF16 storage against FP32 on a large
    GPU ensemble (default 2048 trajectories; the sampling error of a 2% check),
    and FP32 against the FP64 oracle on the oracle's 32 trajectories (same seeds;
    all host cores).  Steps [4000, 8000) of each trajectory; standard errors
    from the spread of per-trajectory values."""
    import multiprocessing as mp

    import numpy as np
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    n = args.clones or 2048
    steps, t0, seed = 8000, 4000, 21
    n_orc = 0 if args.no_cpu else 32
    pool, orc_async = None, None
    if n_orc:  # spawned before the first GPU call
        pool = mp.get_context("spawn").Pool(min(len(os.sched_getaffinity(0)), n_orc))
        orc_async = pool.map_async(_chaotic_oracle_drag, [(seed, c, steps) for c in range(n_orc)])
    torch.cuda.set_device(0)
    L.lib()
    series = {}
    for st in ("fp32", "fp16", "bf16"):
        cfg = L.config(**CHAOTIC, collision="cm", storage=st, max_steps=steps, init_amp=0.01)
        e = L.lbm_ensemble_create(cfg, n, seed, torch.cuda.current_stream())
        t = time.time()
        L.lbm_ensemble_step(e, steps)
        d = np.zeros((n, steps))
        L.lbm_ensemble_drag(e, 0, steps, d)
        series[st] = (d[:, t0:], time.time() - t)
        L.lbm_ensemble_destroy(e)

    def ks(a, b):
        a, b = np.sort(a.ravel()), np.sort(b.ravel())
        x = np.concatenate([a, b])
        return float(np.abs(np.searchsorted(a, x, side="right") / a.size
                            - np.searchsorted(b, x, side="right") / b.size).max())

    def compare(d, ref):
        out = {}
        for name, stat in (("mean", np.mean), ("std", np.std)):
            pa, pb = stat(d, axis=1), stat(ref, axis=1)
            se = float(np.sqrt(pa.var(ddof=1) / pa.size + pb.var(ddof=1) / pb.size))
            out[name] = float(stat(d))
            out[f"{name}_rel_dev"] = float((stat(d) - stat(ref)) / abs(stat(ref)))
            out[f"{name}_rel_se"] = se / abs(float(stat(ref)))
        out["ks"] = ks(d, ref)
        for q in (0.99, 0.999):
            out[f"exceed_q{q}"] = float((d > np.quantile(ref, q)).mean())
        return out

    ref = series["fp32"][0]
    report = {st: dict(compare(d, ref), seconds=round(sec, 3)) for st, (d, sec) in series.items()}
    if n_orc:
        o = np.stack(orc_async.get())[:, t0:]
        pool.close()
        half = np.random.default_rng(0).permutation(n_orc)
        report["fp32_vs_fp64_oracle"] = dict(
            compare(ref[:n_orc], o), trajectories=n_orc,
            ks_null_two_oracle_halves=ks(o[half[:n_orc // 2]], o[half[n_orc // 2:]]))
    print(json.dumps({"metric": "long-run drag statistics of the storage formats", "trajectories": n,
                      "steps": steps, "window": [t0, steps],
                      "config": {"workload": "chaotic open channel 129x33, square R=8, bars R/2 every R, sponge 32, "
                                             "central moments, tau=0.5015, u_c=0.08"},
                      "report": report}))


# ---------------------------------------------------------------- time to return time
def run_return_time(args):
    """Wall time for a return-time estimate of extreme time-averaged drag at 20%
    relative error, plain FP32 direct sampling against the batched GKTL form
    (FP32, FP32 + learned potential, FP16 storage + learned potential).

    Workload (--rt-channel open, the default): the turbulent open channel of
    Sec. 2 (the open workload: 64 trajectories of 513 x 129, central moments,
    tau 0.501), where perturbed clones separate as the paper's cloning
    assumes.  Every replica is a fresh ensemble spun up for 15000 steps (not
    timed), then T_a = T = 20000 steps (10 tau_c) with cloning every 1000
    steps (tau_c / 2), the averaging window equal to the horizon as in the
    paper's GKTL experiments, so that the tilted integral is T F_T.  The
    network of the learned potential sees 64 x 256 blocks of 2 x 2 nodes (the
    outlet column and the top row are past the last whole block).
    --rt-channel periodic: the GKTL ensemble (64 clones of 1024 x 256, 32 x 32
    obstacle, tau 0.505, g_x 1e-6) after a 2000-step spin-up, T_a = T = 10000
    steps, cloning every 500 steps, the network on 4 x 4 blocks.

    Levels a = mean + z sigma of F_T (z = 2, 3, 4) from the direct runs.  For
    each level the GKTL runs are tilted towards it, as the paper chooses k for
    the extremes of interest: k sigma_I = z with sigma_I the spread of the
    integral over the direct runs, which centres the tilted F_T near the level
    for a Gaussian integral.  The direct estimate's relative error is binomial
    at its own estimate (all replicas pooled); where the direct runs saw no
    event its time is a lower bound from the GKTL estimate of P.  The GKTL
    error is measured over independent replicas (at least 16 per variant and
    level).  A variant is credited only if its estimate at z = 2 agrees with
    direct sampling within two combined standard errors.  Wall time to 20% =
    seconds per replica x (relative error / 0.2)^2.  The learned score is
    trained on --rt-snapshots states (default 10^5) of a run of its own, with
    the last tenth held out for its R^2.  Every ensemble is autotuned before it
    is stepped.  --perturbation centred gives every replica the centred App. D
    coefficients (lbm_ensemble_set_perturbation)."""
    import math

    import numpy as np
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    open_ch = args.rt_channel == "open"
    if open_ch:  # the paper's turbulent channel (Sec. 2) with its production collision
        w = workload(argparse.Namespace(workload="open", clones=args.clones or 64, collision=args.collision))
        nx, ny, n, obst = w["nx"], w["ny"], w["clones"], w["obst"]
        chan = dict(channel_kwargs(w), collision=w["collision"])
        spin, t_a, periods, period = 15000, 20000, 20, 1000
    else:
        w = WORKLOADS["gktl"]
        nx, ny, n = w["nx"], w["ny"], w["clones"]
        obst = (nx // 4 - w["side"] // 2, ny // 2 - w["side"] // 2, w["side"], w["side"])
        chan = dict(tau=TAU, gx=GX)
        spin, t_a, periods, period = 2000, 10000, 20, PERIOD
    window = t_a
    R = max(16, args.steps)
    stream = torch.cuda.current_stream()
    factor, rho_s, u_s = (2 if open_ch else 4), 1000.0, 50.0
    zs = (2.0, 3.0, 4.0)

    def make(storage, seed, extra=0):
        cfg = L.config(nx, ny, obstacle=obst, max_steps=spin + t_a + extra, n_snapshots=N_SNAP, storage=storage,
                       **chan)
        return L.lbm_ensemble_create(cfg, n, seed, stream)

    # learned score, trained on an ensemble run of its own (cost reported)
    torch.cuda.synchronize()
    t_train = time.perf_counter()
    H, W = ny // factor, nx // factor
    m = L.cnn_create(H, W, 256, 1)
    every, horizon = 250, 2000
    n_snaps = -(-args.rt_snapshots // n)
    e = make("fp32", 777, extra=(n_snaps - 1) * every + horizon)
    L.lbm_ensemble_autotune(e)
    L.lbm_ensemble_step(e, spin)
    x = torch.zeros((n_snaps * n, H, W, 8), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(n_snaps * n, dtype=torch.float32, device="cuda")
    L.lbm_surrogate_dataset(e, n_snaps, every, horizon, factor, rho_s, u_s, x, y, n, nx, ny)
    L.lbm_ensemble_destroy(e)
    n_tr = (n_snaps - max(1, n_snaps // 10)) * n  # the last tenth of the snapshot times is held out
    losses = L.cnn_fit(m, x[:n_tr], y[:n_tr], 256, args.rt_epochs, 1e-3, 3)
    pred = torch.zeros(n_snaps * n - n_tr, dtype=torch.float32, device="cuda")
    L.cnn_predict(m, x[n_tr:], pred)
    yv = y[n_tr:].double()
    r2_held_out = float(1.0 - ((pred.double() - yv) ** 2).mean() / yv.var(unbiased=False))
    del x, y, pred
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train

    def replica(storage, k, kappa, learned, seed):
        e = make(storage, seed)
        L.lbm_ensemble_autotune(e)
        L.lbm_ensemble_set_perturbation(e, args.perturbation == "centred")
        if learned:
            L.lbm_ensemble_attach_score(e, m, factor, rho_s, u_s)
        L.lbm_ensemble_step(e, spin)
        L.lbm_ensemble_set_snapshots(e, list(range(N_SNAP)))
        logR = torch.zeros(periods, dtype=torch.float64, device="cuda")
        parent = torch.zeros(periods * n, dtype=torch.int32, device="cuda")
        integ = torch.zeros(n, dtype=torch.float64, device="cuda")
        maxima = torch.zeros(n, dtype=torch.float64, device="cuda")
        corr = torch.zeros(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.lbm_gktl_run(e, period, periods, k, EPS, seed, window, logR, parent, integ, maxima,
                       kappa=kappa, correction_dev=corr, refresh_snapshots=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        par = parent.cpu().numpy().reshape(periods, n)
        anc = np.arange(n)
        for i in range(periods - 1, -1, -1):
            anc = par[i][anc]
        L.lbm_ensemble_destroy(e)
        return dict(dt=dt, logR=logR, integ=integ, maxima=maxima, corr=corr, k=k, ancestors=len(set(anc.tolist())))

    direct = [replica("fp32", 0.0, 0.0, False, 100 + r) for r in range(R)]
    F = torch.cat([d["maxima"] for d in direct]).cpu().numpy()
    I = torch.cat([d["integ"] for d in direct]).cpu().numpy()
    mu, sd, sd_i = float(F.mean()), float(F.std()), float(I.std())
    levels = [mu + z * sd for z in zs]
    p_gauss = [0.5 * math.erfc(z / math.sqrt(2.0)) for z in zs]
    variants = {"fp32_gktl": ("fp32", 0.0, False), "fp32_gktl_learned": ("fp32", 0.5, True),
                "fp16_gktl_learned": ("fp16", 0.5, True)}
    # runs[name][j]: the replicas whose estimate serves level j (the direct
    # runs serve every level; GKTL runs are tilted towards their level)
    runs = {"plain_fp32_direct": [direct] * len(zs)}
    for name, (st, kappa, learned) in variants.items():
        runs[name] = [[replica(st, z / sd_i, kappa, learned, 200 + 100 * jz + r) for r in range(R)]
                      for jz, z in enumerate(zs)]
    L.cnn_destroy(m)
    lv = torch.tensor(levels, dtype=torch.float64, device="cuda")
    est = {}  # name -> per level: (estimates per replica, seconds per replica)
    for name, per in runs.items():
        est[name] = []
        for j in range(len(zs)):
            ps = []
            for d in per[j]:
                p = torch.zeros(len(levels), dtype=torch.float64, device="cuda")
                L.gktl_probability(d["k"], d["logR"], d["integ"], d["maxima"], lv, float(t_a), float(window), p,
                                   correction_dev=d["corr"])
                ps.append(float(p[j]))
            est[name].append((np.array(ps), float(np.mean([d["dt"] for d in per[j]]))))
    # direct sampling: the frequency over every trajectory of every replica
    p_direct = [float(ps.mean()) for ps, _ in est["plain_fp32_direct"]]
    se_direct = [math.sqrt(p * (1 - p) / (R * n)) for p in p_direct]
    # a variant is credited only where its z = 2 estimate agrees with direct sampling
    consistent = {}
    for name in variants:
        ps = est[name][0][0]
        se = float(ps.std(ddof=1) / math.sqrt(len(ps)))
        consistent[name] = bool(abs(float(ps.mean()) - p_direct[0]) <= 2 * math.sqrt(se ** 2 + se_direct[0] ** 2))
    out = {}
    for name in runs:
        per_level = []
        for j, z in enumerate(zs):
            ps, t_rep = est[name][j]
            mean = float(ps.mean())
            note = None
            if name == "plain_fp32_direct":
                p_ref = mean
                if mean == 0.0:  # no event: the time is a lower bound, at the credited GKTL estimate of P
                    ok = [float(est[v][j][0].mean()) for v in variants if consistent[v] and est[v][j][0].mean() > 0]
                    p_ref = float(np.mean(ok)) if ok else 0.0
                    note = "no direct event; time at the GKTL estimate of P (a lower bound)"
                cv = binomial_cv(p_ref, n)
            else:
                cv = float(ps.std(ddof=1) / mean) if mean > 0 else float("inf")
            need = seconds_to_rel_error(1.0, cv)
            sec = t_rep * need
            per_level.append({"z": z, "level": levels[j], "k_sigma_I": z if name != "plain_fp32_direct" else 0.0,
                              "P_mean": mean, "P_gauss": p_gauss[j], "replicas": int(len(ps)),
                              "replicas_reaching": int((ps > 0).sum()),
                              "relative_error_per_replica": cv if math.isfinite(cv) else None,
                              "seconds_per_replica": t_rep,
                              "seconds_to_20pct": sec if math.isfinite(sec) else None, "note": note,
                              "distinct_ancestors_mean": float(np.mean([d["ancestors"] for d in runs[name][j]])),
                              # one window per trajectory: waiting time in windows of T steps
                              "return_time_steps": (-window / math.log1p(-mean)) if 0 < mean < 1 else None})
        out[name] = {"levels": per_level}
        if name in variants:
            out[name]["consistent_with_direct_at_z2"] = consistent[name]

    def secs(name, j):
        v = out[name]["levels"][j]["seconds_to_20pct"]
        return v if v is not None else float("inf")
    j3 = len(zs) - 1
    credited = [v for v in variants if consistent[v]]
    plain = secs("plain_fp32_direct", j3)
    best_name = min(credited, key=lambda v: secs(v, j3)) if credited else None
    best = secs(best_name, j3) if best_name else float("inf")
    # what the learned potential costs or gains against plain FP32 GKTL, per level
    learned_factor = {v: {str(z): (secs(v, j) / secs("fp32_gktl", j)
                                   if math.isfinite(secs(v, j)) and math.isfinite(secs("fp32_gktl", j)) else None)
                          for j, z in enumerate(zs)} for v in ("fp32_gktl_learned", "fp16_gktl_learned")}
    print(json.dumps({
        "metric": "time to a 20%-accurate return-time estimate of extreme time-averaged drag",
        "value": best if math.isfinite(best) else None, "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "steps": R, "warmup": 0,
        "data": "synthetic", "dtype": "per variant",
        "config": {"workload": f"GKTL batched ensemble: N={n} clones, {nx}x{ny} "
                               f"{'open channel of Sec. 2' if open_ch else 'periodic channel'}, T_a=T={t_a} steps, "
                               f"cloning every {period} steps, k sigma_I = z for level mean + z sigma of F_T, "
                               f"z = {zs}, eps={EPS}, spin-up {spin} steps", "channel": args.rt_channel,
                   "perturbation": args.perturbation,
                   "replicas": R, "sigma_I": sd_i, "F_T_mean": mu, "F_T_std": sd},
        "variants": out, "best_variant_at_highest_level": best_name, "credited_variants": credited,
        "direct_P_per_level": p_direct,
        "speedup_vs_plain_at_highest_level": (plain / best) if math.isfinite(best) and math.isfinite(plain) else None,
        "speedup_vs_plain_per_level": {
            str(z): (secs("plain_fp32_direct", j) / min(secs(v, j) for v in credited))
            if credited and math.isfinite(secs("plain_fp32_direct", j))
            and math.isfinite(min(secs(v, j) for v in credited)) else None for j, z in enumerate(zs)},
        "learned_vs_fp32_gktl_time_factor": learned_factor,
        "surrogate_training": {"seconds": t_train, "samples": n_tr, "held_out": n_snaps * n - n_tr,
                               "epochs": len(losses), "loss_first_last": [float(losses[0]), float(losses[-1])],
                               "r2_held_out": r2_held_out}}))


# ---------------------------------------------------------------- App. D perturbation against direct sampling
def run_perturbation_bias(args):
    """GKTL's estimate of P(F_T >= mu + 2 sigma) on the open channel of Sec. 2
    against direct sampling, for the App. D perturbation as printed
    (coefficients alpha_n uniform in [0, 1), eps = 0.0002, 0.002, 0.02) and with
    centred coefficients (alpha_n - 1/2, eps = 0.002, 0.02).

    The set-up of the return-time workload: 64 trajectories of 513 x 129, a
    15000-step spin-up per replica, T_a = T = 20000 steps, cloning every 1000
    steps, the App. D bank refilled before each cloning, k sigma_I = 2.  The
    direct arm (k = 0, seeds 100 + r) gives the level and sigma_I; every GKTL
    arm runs the replicas of seeds 200 + r (the seeds of the return-time
    workload's FP32 GKTL at z = 2).  R = max(16, --steps) replicas per arm.
    The direct standard error is given both binomial (all trajectories
    independent) and from the spread of the replicas' frequencies."""
    import math

    import numpy as np
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    w = workload(argparse.Namespace(workload="open", clones=args.clones or 64, collision=args.collision))
    nx, ny, n, obst = w["nx"], w["ny"], w["clones"], w["obst"]
    chan = dict(channel_kwargs(w), collision=w["collision"])
    spin, t_a, periods, period, z = 15000, 20000, 20, 1000, 2.0
    R = max(16, args.steps)
    stream = torch.cuda.current_stream()

    def replica(k, eps, centred, seed):
        cfg = L.config(nx, ny, obstacle=obst, max_steps=spin + t_a, n_snapshots=N_SNAP, storage="fp32", **chan)
        e = L.lbm_ensemble_create(cfg, n, seed, stream)
        L.lbm_ensemble_autotune(e)
        L.lbm_ensemble_set_perturbation(e, centred)
        L.lbm_ensemble_step(e, spin)
        L.lbm_ensemble_set_snapshots(e, list(range(N_SNAP)))
        logR = torch.zeros(periods, dtype=torch.float64, device="cuda")
        parent = torch.zeros(periods * n, dtype=torch.int32, device="cuda")
        integ = torch.zeros(n, dtype=torch.float64, device="cuda")
        maxima = torch.zeros(n, dtype=torch.float64, device="cuda")
        L.lbm_gktl_run(e, period, periods, k, eps, seed, t_a, logR, parent, integ, maxima, refresh_snapshots=True)
        par = parent.cpu().numpy().reshape(periods, n)
        anc = np.arange(n)
        for i in range(periods - 1, -1, -1):
            anc = par[i][anc]
        L.lbm_ensemble_destroy(e)
        return dict(logR=logR, integ=integ, maxima=maxima, ancestors=len(set(anc.tolist())))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    direct = [replica(0.0, EPS, False, 100 + r) for r in range(R)]
    F = np.stack([d["maxima"].cpu().numpy() for d in direct])
    I = np.stack([d["integ"].cpu().numpy() for d in direct])
    mu, sd, sd_i = float(F.mean()), float(F.std()), float(I.std())
    level = mu + z * sd
    freq = (F >= level).mean(axis=1)
    p_dir = float(freq.mean())
    se_bin = math.sqrt(p_dir * (1 - p_dir) / F.size)
    se_rep = float(freq.std(ddof=1) / math.sqrt(R))
    lv = torch.tensor([level], dtype=torch.float64, device="cuda")
    k = z / sd_i
    arms = []
    for centred, eps in ((False, 0.0002), (False, EPS), (False, 0.02), (True, EPS), (True, 0.02)):
        ps, anc = [], []
        for r in range(R):
            d = replica(k, eps, centred, 200 + r)
            p = torch.zeros(1, dtype=torch.float64, device="cuda")
            L.gktl_probability(k, d["logR"], d["integ"], d["maxima"], lv, float(t_a), float(t_a), p)
            ps.append(float(p[0]))
            anc.append(d["ancestors"])
        ps = np.array(ps)
        se = float(ps.std(ddof=1) / math.sqrt(R))
        arms.append({"coefficients": "centred alpha_n - 1/2" if centred else "uniform [0, 1) (printed)", "eps": eps,
                     "P_mean": float(ps.mean()), "P_median": float(np.median(ps)), "standard_error": se,
                     "ratio_to_direct": float(ps.mean()) / p_dir if p_dir > 0 else None,
                     "standard_errors_from_direct": (float(ps.mean()) - p_dir) / math.sqrt(se ** 2 + se_bin ** 2),
                     "distinct_ancestors_mean": float(np.mean(anc)), "per_replica": ps.tolist()})
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    print(json.dumps({
        "metric": "GKTL estimate of P(F_T >= mean + 2 std) against direct sampling, by App. D perturbation",
        "value": arms[-2]["ratio_to_direct"], "unit": "ratio to direct sampling (centred, eps 0.002)",
        "higher_is_better": None, "n_gpus": 1, "steps": R, "warmup": 0, "data": "synthetic", "dtype": "f32",
        "seconds": seconds,
        "config": {"workload": f"open channel of Sec. 2, N={n} trajectories of {nx}x{ny}, spin-up {spin} steps, "
                               f"T_a=T={t_a} steps, cloning every {period} steps, k sigma_I = {z:g}",
                   "replicas_per_arm": R, "F_T_mean": mu, "F_T_std": sd, "sigma_I": sd_i, "level": level},
        "direct": {"P": p_dir, "standard_error_binomial": se_bin, "standard_error_replicas": se_rep,
                   "trajectories": int(F.size)},
        "gktl": arms}))


# ---------------------------------------------------------------- CNN
def cnn_flops_per_sample(H, W, train: bool) -> float:
    """algorithmic FLOPs of the surrogate on one H x W input (3 real input
    channels): 2 x pixels x 32 x taps per conv layer; training adds the weight
    gradient of every layer and the data gradient of layers 1..3"""
    P = H * W
    fwd = 2 * P * 32 * (9 * 3) + 3 * 2 * P * 32 * (9 * 32)
    if not train:
        return fwd
    return fwd + fwd + 3 * 2 * P * 32 * (9 * 32)


def run_cnn(args):
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    H, W, B = 64, 256, 256
    m = L.cnn_create(H, W, B, 1)
    stream = torch.cuda.current_stream()
    x = torch.zeros((B, H, W, 8), device="cuda")
    x[..., :3] = torch.randn((B, H, W, 3), device="cuda")
    x = x.to(torch.bfloat16).contiguous()
    y = torch.randn(B, device="cuda")
    pred = torch.zeros(B, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(args.warmup):
        L.cnn_forward(m, x, pred, stream)
        L.cnn_train_step(m, x, y, 1e-4, None, stream)
    torch.cuda.synchronize()
    launches0 = L.lbm_launch_count()
    ev[0].record(stream)
    for _ in range(args.steps):
        L.cnn_forward(m, x, pred, stream)
    ev[1].record(stream)
    for _ in range(args.steps):
        L.cnn_train_step(m, x, y, 1e-4, None, stream)
    ev[2].record(stream)
    torch.cuda.synchronize()
    launches = L.lbm_launch_count() - launches0
    fwd_ms = ev[0].elapsed_time(ev[1]) / args.steps
    trn_ms = ev[1].elapsed_time(ev[2]) / args.steps
    L.cnn_destroy(m)
    fwd_tf = cnn_flops_per_sample(H, W, False) * B / (fwd_ms / 1e3) / 1e12
    trn_tf = cnn_flops_per_sample(H, W, True) * B / (trn_ms / 1e3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, kind = float(json.load(fh)["bf16_tflops"]), "measured bf16_tflops (burst)"
    except Exception:
        peak, kind = 1900.0, "fallback"
    print(json.dumps({
        "metric": "learned-score CNN throughput", "value": B / (trn_ms / 1e3), "unit": "training samples/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": trn_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": f"CNN 4x conv3x3 32 ch on {H}x{W} inputs (4x-downsampled 1024x256), batch {B}"},
        "forward": {"ms_per_batch": fwd_ms, "samples_per_s": B / (fwd_ms / 1e3), "tflops": fwd_tf},
        "train": {"ms_per_batch": trn_ms, "tflops": trn_tf},
        "roofline": {"bound": "tensor", "achieved": trn_tf, "peak": peak, "unit": "TFLOP/s", "frac": trn_tf / peak,
                     "traffic": None, "peak_kind": kind},
        "gpu_launches": launches}))


def run_ams_branch(args):
    """The AMS branching phase (App. B.1): after a kill, one trajectory is
    restarted and stepped alone to T_a, in chunks cut by its checkpoints.  One
    bench step = one branch of 2000 lattice steps of one 512x128 trajectory of
    the AMS workload with a checkpoint every 250 steps, taken in turn from a
    pool of 16 trajectories; timed with step-chunk graphs (the default) and
    with one direct launch per lattice step.  --ams-channel open: the same on
    one trajectory of the open channel of Sec. 2 (its outlet column written by a
    second kernel at the end of each chunk)."""
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    open_ch = args.ams_channel == "open"
    if open_ch:  # the paper's channel (Sec. 2) with its production collision
        w = workload(argparse.Namespace(workload="open", clones=16, collision=args.collision))
        chan = dict(channel_kwargs(w), collision=w["collision"])
    else:
        w = workload(argparse.Namespace(workload="ams", clones=16))
        chan = dict(tau=TAU, gx=GX)
    n, branch, stride = 16, 2000, 250
    modes = [("graphs", True), ("direct", False)]
    if len(modes) * (args.steps + args.warmup) > n * (10000 // branch):
        raise SystemExit(f"ams-branch: at most {n * (10000 // branch) // len(modes)} steps + warm-up")
    stream = torch.cuda.current_stream()
    cfg = L.config(w["nx"], w["ny"], obstacle=w["obst"], storage=L.STORAGE[args.storage], max_steps=10000,
                   ckpt_stride=stride, **chan)
    e = L.lbm_ensemble_create(cfg, n, 1, stream)
    if args.variant != "auto":
        L.lbm_ensemble_set_variant(e, int(args.variant))
    nxt = [0]

    def one_branch():
        c = nxt[0] % n
        nxt[0] += 1
        L.lbm_ensemble_step_clones(e, branch, [c])

    res = {}
    launches = 0
    for mode, graphs in modes:
        L.lbm_ensemble_set_graphs(e, graphs)
        for _ in range(args.warmup):
            one_branch()
        torch.cuda.synchronize()
        l0 = L.lbm_launch_count()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(args.steps):
            one_branch()
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / args.steps
        res[mode] = ms
        if mode == "graphs":
            launches = L.lbm_launch_count() - l0
    L.lbm_ensemble_destroy(e)
    sites = w["nx"] * w["ny"]
    glups = {g: sites * branch / (ms / 1e3) / 1e9 for g, ms in res.items()}
    bps = BYTES_PER_SITE if args.storage == "fp32" else BYTES_PER_SITE // 2
    hbm, peak_kind = peaks()
    achieved = bps * sites * branch / (res["graphs"] / 1e3) / 1e9
    print(json.dumps({
        "metric": "AMS branch-phase stepping rate (one trajectory)", "value": glups["graphs"], "unit": "GLUPS",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["graphs"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"AMS branch: one {w['nx']}x{w['ny']} trajectory ({args.storage}), {branch} lattice "
                               f"steps per bench step, checkpoint every {stride} steps, pool of {n}",
                   "storage": args.storage, "channel": args.ams_channel,
                   "l2": "working set of one trajectory (two buffers) is L2-resident; no flush: this is the "
                         "branch phase as AMS runs it"},
        "direct_launches": {"value": glups["direct"], "unit": "GLUPS", "ms_per_step": res["direct"],
                            "us_per_lattice_step": 1e3 * res["direct"] / branch},
        "graphs": {"us_per_lattice_step": 1e3 * res["graphs"] / branch, "speedup": res["direct"] / res["graphs"]},
        "roofline": {"bound": "latency", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "peak_kind": f"{peak_kind} hbm_gbs; algorithmic bytes of an L2-resident "
                                                   f"working set, so frac may exceed 1"},
        "gpu_launches": launches}))


def run_ams_run(args):
    """A whole AMS run (App. B.1) on the AMS workload: N trajectories of
    512x128 stepped to T_a, then kill-and-branch iterations (each restores the
    survivor's checkpoint, replays to the branching time, perturbs with the
    App. D bank refilled from that checkpoint and steps the copy to T_a).  The
    score is the instantaneous drag (--ams-window 1, the paper's Sec. 4.1
    workload) or its trailing mean.  One bench step = one run on a fresh
    ensemble; reported: milliseconds per run, with the initial ensemble timed
    on its own."""
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    open_ch = args.ams_channel == "open"
    if open_ch:  # the paper's channel (Sec. 2) with its production collision
        w = workload(argparse.Namespace(workload="open", clones=args.clones or 256, collision=args.collision))
        chan = dict(channel_kwargs(w), collision=w["collision"])
    else:
        w = workload(argparse.Namespace(workload="ams", clones=args.clones))
        chan = dict(tau=TAU, gx=GX)
    n, t_a, J, stride = w["clones"], 2000, 40, 250
    window = args.ams_window
    stream = torch.cuda.current_stream()
    cfg = L.config(w["nx"], w["ny"], obstacle=w["obst"], storage=L.STORAGE[args.storage], max_steps=t_a,
                   ckpt_stride=stride, n_snapshots=N_SNAP, **chan)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    runs, inits, iters, launches = [], [], [], 0
    for step in range(args.warmup + args.steps):
        e = L.lbm_ensemble_create(cfg, n, 2000 + step, stream)
        try:
            L.lbm_ensemble_set_snapshots(e, [i * n // N_SNAP for i in range(N_SNAP)])
            Q = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            l0 = L.lbm_launch_count()
            ev[0].record(stream)
            it, lw, levels = L.lbm_ams_run(e, t_a, window, J, float("inf"), EPS, 7 + step, Q,
                                           refresh_snapshots=True)
            ev[1].record(stream)
            torch.cuda.synchronize()
            l1 = L.lbm_launch_count()
        finally:
            L.lbm_ensemble_destroy(e)
        e = L.lbm_ensemble_create(cfg, n, 2000 + step, stream)  # the initial ensemble alone
        try:
            torch.cuda.synchronize()
            ev[2].record(stream)
            L.lbm_ensemble_step(e, t_a)
            ev[3].record(stream)
            torch.cuda.synchronize()
        finally:
            L.lbm_ensemble_destroy(e)
        if step >= args.warmup:
            runs.append(ev[0].elapsed_time(ev[1]))
            inits.append(ev[2].elapsed_time(ev[3]))
            iters.append(it)
            launches += l1 - l0
    ms = statistics.median(runs)
    init_ms = statistics.median(inits)
    it_med = statistics.median(iters)
    score = "instantaneous drag" if window == 1 else f"{window}-step time-averaged drag"
    print(json.dumps({
        "metric": "AMS run time (initial ensemble + kill/branch iterations)", "value": ms, "unit": "ms per run",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"AMS: N={n} trajectories of {w['nx']}x{w['ny']} "
                               f"{'open channel of Sec. 2, ' + w['collision'] + ' collision, ' if open_ch else ''}"
                               f"({args.storage}), T_a={t_a}, "
                               f"up to {J} iterations, score = {score}, checkpoints every {stride} steps, "
                               f"App. D bank of {N_SNAP} refilled at each branch",
                   "storage": args.storage, "score_window": window, "channel": args.ams_channel},
        "initial_ensemble": {"ms": init_ms, "glups": n * w["nx"] * w["ny"] * t_a / (init_ms / 1e3) / 1e9},
        "branch_phase": {"iterations": it_med, "ms_per_iteration": (ms - init_ms) / max(it_med, 1)},
        "gpu_launches": launches // max(len(runs), 1)}))


def run_ams_estimate(args):
    """Seconds to a 20%-accurate estimate of P(max_t D(t) >= a), the extreme
    instantaneous drag of Sec. 4.1, by AMS (App. B.1) against direct sampling,
    on the open channel of Sec. 2 (central moments, tau 0.501).

    Every run is a fresh ensemble of N = 32 trajectories spun up for 15000
    steps (not timed); T_a = 2000 steps (about tau_c), score = the
    instantaneous drag, checkpoints every 250 steps, App. D bank refilled at
    each branch.  Direct sampling: runs with no iteration give the maxima Q of
    N independent trajectories; levels a = mean + z sigma of Q (z = 2, 3, 4).
    AMS: per level, runs that kill until the level is reached (at most 40 N
    iterations); the generalized-AMS estimate is exp(log weight) x the
    fraction of final maxima >= a, its relative error the spread over runs.
    The direct-sampling error is binomial at the AMS mean (the unbiased
    estimate of p).  Seconds to 20% = seconds per run x (relative error / 0.2)^2,
    a direct run being N trajectories."""
    import math

    import numpy as np
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    w = workload(argparse.Namespace(workload="open", clones=args.clones or 32, collision=args.collision))
    n, spin, t_a, stride = w["clones"], 15000, 2000, 250
    R = max(3, args.steps)
    stream = torch.cuda.current_stream()
    cfg = L.config(w["nx"], w["ny"], obstacle=w["obst"], storage=L.STORAGE[args.storage], max_steps=spin + t_a,
                   ckpt_stride=stride, n_snapshots=N_SNAP, collision=w["collision"], **channel_kwargs(w))
    zs = (2.0, 3.0, 4.0)

    def run(seed, level, max_iter):
        e = L.lbm_ensemble_create(cfg, n, seed, stream)
        try:
            L.lbm_ensemble_autotune(e)
            L.lbm_ensemble_step(e, spin)
            L.lbm_ensemble_set_snapshots(e, [i * n // N_SNAP for i in range(N_SNAP)])
            Q = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, lw, _ = L.lbm_ams_run(e, t_a, 1, max_iter, level, EPS, seed, Q, refresh_snapshots=True)
            torch.cuda.synchronize()
            return time.perf_counter() - t0, it, lw, Q.cpu().numpy()
        finally:
            L.lbm_ensemble_destroy(e)

    direct = [run(500 + r, float("inf"), 0) for r in range(2 * R)]
    Qd = np.concatenate([d[3] for d in direct])
    t_direct = float(np.mean([d[0] for d in direct]))  # one run = N trajectories
    mu, sd = float(Qd.mean()), float(Qd.std())
    levels = []
    for z in zs:
        a = mu + z * sd
        rs = [run(700 + 100 * int(z) + r, a, 40 * n) for r in range(R)]
        ps = np.array([ams_estimate(lw, Q, a) for _, _, lw, Q in rs])
        p = float(ps.mean())
        t_run = float(np.mean([r[0] for r in rs]))
        cv = float(ps.std(ddof=1) / p) if p > 0 else float("inf")
        p_dir = float((Qd >= a).mean())
        cv_dir = binomial_cv(p, n)
        levels.append({"z": z, "level": a, "P_ams": p, "P_direct_sample": p_dir,
                       "direct_events": int((Qd >= a).sum()), "direct_trajectories": int(Qd.size),
                       "ams_iterations_mean": float(np.mean([r[1] for r in rs])),
                       "ams_runs_reaching": int((ps > 0).sum()), "ams_relative_error_per_run": cv,
                       "ams_seconds_per_run": t_run, "ams_seconds_to_20pct": seconds_to_rel_error(t_run, cv),
                       "direct_seconds_per_run": t_direct,
                       "direct_seconds_to_20pct": seconds_to_rel_error(t_direct, cv_dir),
                       "speedup": (t_direct * cv_dir ** 2) / (t_run * cv ** 2) if cv > 0 and p > 0 else None,
                       "return_time_steps": (-t_a / math.log1p(-p)) if 0 < p < 1 else None})
    top = levels[-1]
    print(json.dumps({
        "metric": "time to a 20%-accurate estimate of P(max instantaneous drag >= a), AMS vs direct sampling",
        "value": top["ams_seconds_to_20pct"], "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": R,
        "warmup": 0, "data": "synthetic", "dtype": args.storage,
        "config": {"workload": f"AMS (App. B.1) on the open channel of Sec. 2: N={n} trajectories of "
                               f"{w['nx']}x{w['ny']}, {w['collision']} collision, spin-up {spin} steps, T_a={t_a}, "
                               f"score = instantaneous drag, checkpoints every {stride} steps; levels mean + z sigma "
                               f"of the direct maxima, z = {zs}", "runs_per_level": R, "direct_runs": 2 * R,
                   "Q_mean": mu, "Q_std": sd},
        "levels": levels}))


def solid_cells(w) -> int:
    """solid cells of the workload's channel: the square and, in the open
    channel, the entrance grid's bars (rows with y mod (bar + gap) >= gap over
    the grid's columns)"""
    n = w["obst"][2] * w["obst"][3]
    if w.get("open"):
        _, width, bar, gap = OPEN_GRID
        n += width * sum(1 for y in range(w["ny"]) if y % (bar + gap) >= gap)
    return n


def binomial_cv(p: float, n: int) -> float:
    """relative error of a direct-sampling frequency of probability p over n
    independent samples (inf unless 0 < p < 1)"""
    import math
    return math.sqrt((1.0 - p) / (n * p)) if 0.0 < p < 1.0 else float("inf")


def seconds_to_rel_error(seconds_per_run: float, cv_per_run: float, target: float = 0.2) -> float:
    """wall time for independent runs to average to a relative error `target`:
    the error of a mean of m runs is cv / sqrt(m)"""
    return seconds_per_run * (cv_per_run / target) ** 2


def ams_estimate(log_weight: float, maxima, level: float) -> float:
    """generalized-AMS estimate of P(max score >= level) from one run (App.
    B.1): the product of the survival fractions (1 - K_j / N), exp(log_weight),
    times the fraction of the final ensemble's maxima at or above the level"""
    import math

    import numpy as np
    return math.exp(log_weight) * float((np.asarray(maxima) >= level).mean())


def ks_distance(a, b) -> float:
    """two-sample Kolmogorov-Smirnov distance of the empirical distributions"""
    import numpy as np
    a, b = np.sort(np.ravel(a)), np.sort(np.ravel(b))
    grid = np.concatenate([a, b])
    return float(np.max(np.abs(np.searchsorted(a, grid, side="right") / len(a)
                               - np.searchsorted(b, grid, side="right") / len(b))))


def pooled_tau_c(x, max_lag: int) -> int:
    """first lag at which the autocorrelation pooled over the rows of x is <= 0
    (the correlation time of Sec. 3; -1 if none within max_lag); the lagged
    sums by FFT, each lag divided by its number of products"""
    import numpy as np
    x = x - x.mean()
    n = x.shape[1]
    m = 1 << int(np.ceil(np.log2(2 * n)))
    spec = np.fft.rfft(x, m, axis=1)
    acf = np.fft.irfft(spec * np.conj(spec), m, axis=1)[:, :max_lag + 1].sum(axis=0)
    acf /= x.shape[0] * (n - np.arange(max_lag + 1))
    below = np.nonzero(acf[1:] <= 0.0)[0]
    return int(below[0]) + 1 if len(below) else -1


def run_perturb_check(args):
    """The paper's check that the App. D perturbation leaves the drag statistics
    unchanged: on the open channel of Sec. 2 (the open workload), half of the
    trajectories are perturbed in place (eps = 0.002, 10 snapshots) every
    --check-period steps, the other half run unperturbed, and the square's
    observables are recorded after every step.  The default period, 1000 steps,
    is tau_c / 2 of the developed flow's drag (tau_c about 2060 steps over
    steps 15000-65000).
    The App. D bank holds flow states of the unperturbed half, refilled when
    the warm-up (the spin-up of the channel) ends.
    One bench step = CHECK_STEPS lattice steps of the whole ensemble, the
    perturbations and the observables included.  Reported: GLUPS, and the
    statistics of each half over the timed steps, with the KS distance between
    the halves against that between the two quarters of the unperturbed half
    (a null reference of the same sample size).  --perturbation centred
    perturbs with centred App. D coefficients."""
    import numpy as np
    import torch

    from paper_2005_09323_gb300 import lbmrare as L
    torch.cuda.set_device(0)
    L.lib()
    w = workload(argparse.Namespace(workload="open", clones=args.clones, collision=args.collision))
    n = w["clones"]
    half = list(range(n // 2))
    total = CHECK_STEPS * (args.warmup + args.steps)
    stream = torch.cuda.current_stream()
    cfg = L.config(w["nx"], w["ny"], obstacle=w["obst"], max_steps=total, n_snapshots=N_SNAP, init_amp=0.01,
                   storage=args.storage, collision=w["collision"], **channel_kwargs(w))
    e = L.lbm_ensemble_create(cfg, n, 31, stream)
    L.lbm_ensemble_set_observables(e, True)
    L.lbm_ensemble_set_perturbation(e, args.perturbation == "centred")
    state = {"it": 0}
    bank = [n // 2 + i * (n // 2) // N_SNAP for i in range(N_SNAP)]  # unperturbed trajectories

    period = args.check_period

    def bench_step():
        for k in range(CHECK_STEPS // period):
            L.lbm_ensemble_step(e, period)
            if state["it"] == 0:  # a first bank for the spin-up
                L.lbm_ensemble_set_snapshots(e, bank)
            L.lbm_ensemble_perturb(e, half, EPS, 11, state["it"])
            state["it"] += 1
        # the remainder of the bench step, unperturbed until the next period
        if CHECK_STEPS % period:
            L.lbm_ensemble_step(e, CHECK_STEPS % period)

    for _ in range(args.warmup):
        bench_step()
    L.lbm_ensemble_set_snapshots(e, bank)  # states of the developed flow
    torch.cuda.synchronize()
    l0 = L.lbm_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            bench_step()
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = L.lbm_launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    t0, t1 = CHECK_STEPS * args.warmup, total
    drag = np.zeros((n, t1 - t0))
    L.lbm_ensemble_drag(e, t0, t1, drag)
    obs = np.zeros((n, t1 - t0, 4))
    L.lbm_ensemble_observables(e, t0, t1, obs)
    L.lbm_ensemble_destroy(e)

    def stats(rows):
        d, o = drag[rows], obs[rows]
        dp = o[..., 0] - o[..., 1]
        return {"clones": len(rows), "drag_mean": float(d.mean()), "drag_std": float(d.std()),
                "tau_c_steps": pooled_tau_c(d, min(20000, d.shape[1] - 1)), "p_fb_minus_p_base_mean": float(dp.mean()),
                "p_fb_minus_p_base_std": float(dp.std()), "gamma_top_mean": float(o[..., 2].mean()),
                "gamma_top_std": float(o[..., 2].std()), "gamma_bottom_mean": float(o[..., 3].mean()),
                "corr_drag_pressure_diff": float(np.corrcoef(d.ravel(), dp.ravel())[0, 1])}

    pert, unpert = half, list(range(n // 2, n))
    q = len(unpert) // 2
    sites = n * w["nx"] * w["ny"]
    print(json.dumps({
        "metric": "Perturbation check (App. D): GLUPS with in-place perturbation and observables",
        "value": sites * CHECK_STEPS * args.steps / (ms / 1e3) / 1e9, "unit": "GLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"Perturbation check (App. D) on the open channel of Sec. 2: N={n} trajectories of "
                               f"{w['nx']}x{w['ny']}, square, grid, sponge, tau={OPEN_TAU:.4f}, {w['collision']} "
                               f"collision, {args.storage}; clones 0..{n // 2 - 1} perturbed in place every "
                               f"{period} steps (eps={EPS}, bank of {N_SNAP} unperturbed states refilled "
                               f"after the {CHECK_STEPS * args.warmup}-step warm-up), the rest unperturbed; "
                               f"observables every step; {CHECK_STEPS} steps per step",
                   "storage": args.storage, "collision": w["collision"]},
        "perturbation_check": {
            "window_steps": [t0, t1], "period_steps": period, "eps": EPS, "coefficients": args.perturbation,
            "perturbed": stats(pert), "unperturbed": stats(unpert),
            "ks_drag_perturbed_vs_unperturbed": ks_distance(drag[pert], drag[unpert]),
            "ks_drag_null_unperturbed_quarters": ks_distance(drag[unpert[:q]], drag[unpert[q:]]),
            "note": "bench-length run from the inlet-profile start; the paper's check ran 1e5 tau_c"},
        "gpu_launches": launches, "clocks": clk.summary()}))


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
    ap.add_argument("--workload", default="gktl", choices=sorted(WORKLOADS) + ["cnn", "return-time", "precision-report", "ams-branch", "ams-run", "ams-estimate",
                                              "perturb-check", "long-run-precision", "perturbation-bias"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--collision", default=None, choices=["bgk", "cm"],
                    help="BGK or the central-moment collision (default: central moments for the open "
                         "channel, BGK otherwise)")
    ap.add_argument("--check-period", type=int, default=CHECK_PERIOD,
                    help="perturb-check: steps between in-place perturbations (the paper: tau_c / 2)")
    ap.add_argument("--ams-channel", default="periodic", choices=["periodic", "open"],
                    help="ams-run: the periodic AMS channel or the paper's open channel")
    ap.add_argument("--rt-channel", default="open", choices=["periodic", "open"],
                    help="return-time workload: the turbulent open channel of Sec. 2 (default) or the periodic "
                         "GKTL channel")
    ap.add_argument("--rt-snapshots", type=int, default=100000,
                    help="return-time workload: flow states the learned score is trained on")
    ap.add_argument("--rt-epochs", type=int, default=20, help="return-time workload: training epochs")
    ap.add_argument("--perturbation", default="printed", choices=["printed", "centred"],
                    help="return-time and perturb-check workloads: App. D coefficients uniform in [0, 1) as "
                         "printed, or centred")
    ap.add_argument("--ams-window", type=int, default=1,
                    help="ams-run: score window in steps (1 = the instantaneous drag)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "cnn":
        run_cnn(args)
    elif args.workload == "return-time":
        run_return_time(args)
    elif args.workload == "precision-report":
        run_precision_report(args)
    elif args.workload == "long-run-precision":
        run_long_run_precision(args)
    elif args.workload == "ams-branch":
        run_ams_branch(args)
    elif args.workload == "ams-estimate":
        run_ams_estimate(args)
    elif args.workload == "ams-run":
        run_ams_run(args)
    elif args.workload == "perturb-check":
        run_perturb_check(args)
    elif args.workload == "perturbation-bias":
        run_perturbation_bias(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

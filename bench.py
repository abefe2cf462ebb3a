"""Benchmark of the two-phase Darcy LB solver (one JSON line on stdout).

Workload (default): the quarter five-spot of 1024 x 1024 nodes (ln K a seeded Gaussian
random field, sigma 1, correlation length 16 cells; no-flux walls; injector and producer
of rate 1e-3 at opposite corners; S0 = 0.2; phi = 0.2, beta = 0.4, mu_w = 1, mu_n = 2,
D_s = 0.01, tau_p = 1, tau_s = 0.8), each physical step sub-iterating the pressure to a
relative increment of 1e-8.  A step = S refresh + pressure sub-iteration + saturation
update.  The t = 0 initialisation (the pressure solve, started from the same problem
solved on a 4x coarser lattice unless --cold-start) is set-up, outside the timing.

Metric: MLUPS = nodes x (pressure sweeps + 1 saturation update) / time, summed over the
timed steps (and over ranks).  L2 is flushed before every timed step; each step is timed
with CUDA events on the solver's stream.

Workload batch_five_spot_64: 64 independent five-spot realisations with sizes drawn from
{128, 256, 512}^2 (sigma, correlation length and viscosity ratio drawn per member), advanced
together by one lbm2p_batch per step; the line also reports the same members stepped one
after another.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload five_spot_1024|five_spot_4096|manufactured_64|batch_five_spot_64]
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

# algorithmic bytes per node of one pressure-sweep launch: 8 populations read and written
# (stored as FP32 deviations) + the reference pressure + 1/tau_f; a launch that fuses T
# sweeps moves the same bytes once for T sweeps
BYTES_PER_SWEEP_NODE = 72
# with FP16 storage: 8 populations x (2 + 2) B + the node pressure read and written + 1/tau_f
BYTES_PER_SWEEP_NODE_FP16 = 44
WORKLOADS = {
    "five_spot_1024": dict(kind="five_spot", n=1024),
    "five_spot_4096": dict(kind="five_spot", n=4096),
    "manufactured_64": dict(kind="manufactured", n=64),
    # independent five-spot realisations of uneven sizes advanced by one batch (lbm2p_batch)
    "batch_five_spot_64": dict(kind="batch", count=64, sizes=(128, 256, 512)),
}
SWEEP_KERNEL_NAMES = {1: "four nodes per thread (128-bit accesses)", 2: "one node per thread",
                      3: "rows staged in shared memory by bulk async copies"}
# DRAM bytes per pressure-sweep launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by workload and launch form (sweeps per launch, fused tile width or single kernel
# kind); absent until captured for the current kernel (profiles/).
# five_spot_1024, one node per thread (the autotuner's choice there): 42.0 MB read + 0.9 MB
# written per launch, L2 flushed by ncu before the launch.
# five_spot_1024, two sweeps with direct loads, 120-column blocks of 4 rows (the autotuner's
# choice there with the residual checked every 16 sweeps): 42.0 MB read + 0.95 MB written per
# launch, L2 flushed by ncu before the launch.
# five_spot_4096, two sweeps on staged rows, 120-column blocks (the autotuner's choice there):
# 720.9 MB read + 493.1 MB written per launch (a launch without the residual).
NCU_TRAFFIC_PER_LAUNCH = {("five_spot_1024", "single", 2): 42.87e6,
                          ("five_spot_1024", "direct", 120): 42.94e6,
                          ("five_spot_4096", "staged_rows", 120): 1214.0e6}
FUSED_FORM_NAMES = {1: "stages", 2: "staged_rows", 3: "direct"}
FUSED_FORM_TEXT = {1: "on shared-memory stages", 2: "on rows staged by bulk copies",
                   3: "with direct loads"}


def batch_members(name: str, rank: int = 0):
    """Realisations of a batch workload: sizes drawn uniformly from the workload's list,
    sigma of ln K in [0.5, 2], correlation length in [8, 32] cells, viscosity ratio
    mu_n / mu_w in [0.5, 10] (mu_w = 1), GRF seeds 4000 + member index."""
    w = WORKLOADS[name]
    rng = np.random.default_rng(4000 + rank)
    out = []
    for r in range(w["count"]):
        n = int(rng.choice(w["sizes"]))
        sigma, corr = float(rng.uniform(0.5, 2.0)), float(rng.uniform(8.0, 32.0))
        ratio = float(rng.uniform(0.5, 10.0))
        out.append(W.quarter_five_spot(n, seed=4000 + rank * w["count"] + r, sigma=sigma,
                                       corr_len=corr, mu_w=1.0, mu_n=ratio))
    return out


def make_problem(name: str, rank: int = 0):
    w = WORKLOADS[name]
    if w["kind"] == "batch":
        return batch_members(name, rank)[0]
    if w["kind"] == "five_spot":
        return W.quarter_five_spot(w["n"], seed=2 + rank)
    return W.manufactured_periodic(w["n"])


def coarse_initial_pressure(prob, pkg, factor=4, min_n=64, log=None):
    """Initial pressure guess for a five-spot from the same problem on a coarser lattice
    (set-up only; the paper leaves the t = 0 guess free).  K is averaged geometrically
    over factor x factor blocks, the wells stay at the corner nodes, dt scales with dx^2;
    the coarse solve itself starts from a still coarser guess, down to min_n nodes, and is
    only converged to a relative increment of 1e-6 (a guess, not a solution)."""
    if prob.wells == [] or prob.nx % factor or prob.ny % factor or prob.nx // factor < min_n:
        return None
    nx, ny = prob.nx // factor, prob.ny // factor
    lnK = np.log(prob.K).reshape(ny, factor, nx, factor).mean(axis=(1, 3))
    c = W.quarter_five_spot(nx, ny, seed=0)
    c.K = np.exp(lnK)
    c.dx, c.dt = prob.dx * factor, prob.dt * factor * factor
    c.mu_w, c.mu_n, c.tau_p = prob.mu_w, prob.mu_n, prob.tau_p
    c.wells = [(0, 0, prob.wells[0][2], 0), (nx - 1, ny - 1, prob.wells[1][2], 1)]
    c.S0 = prob.S0.reshape(ny, factor, nx, factor).mean(axis=(1, 3))
    c.P0 = coarse_initial_pressure(c, pkg, factor, min_n, log)
    s = pkg.Solver.from_problem(c, tol=1e-6, max_sub_iters=200_000)
    if log is not None:
        log.append({"n": nx, "sweeps": s.init_stats.sub_iters, "r": s.init_stats.residual})
    P, _ = s.fields()
    s.close()
    return np.kron(P.astype(np.float64), np.ones((factor, factor)))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples every 20 ms; only samples stamped inside the timed region count
    (start() returns once the first sample has arrived, so the region is covered)."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            deadline = time.time() + 5.0
            while not self.lines and time.time() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                if self.t0 is not None and not (self.t0 <= ts <= self.t1):
                    continue
                sm.append(float(parts[2]))
                smax.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm), "sample_ms": 20}


# ---------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores, bounded sample of the same workload
# ---------------------------------------------------------------------------------------
def cpu_baseline(name: str, budget_s: float = 12.0):
    import oracle as O
    prob = make_problem(name)
    orc = O.Oracle(prob, tol=1e-8, init_replay=0)
    nodes = prob.nx * prob.ny
    # calibrate: one step of 5 sweeps
    t0 = time.perf_counter()
    orc.step(1, replay=[5])
    t1 = time.perf_counter()
    per_update = (t1 - t0) / (nodes * 6)
    sweeps = max(5, int(budget_s / (per_update * nodes)) - 1)
    t0 = time.perf_counter()
    orc.step(1, replay=[sweeps])
    dt = time.perf_counter() - t0
    orc.close()
    updates = nodes * (sweeps + 1)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": updates / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{name}: 1 physical step with {sweeps} pressure sweeps + 1 saturation "
                      f"update on the {prob.nx}x{prob.ny} lattice, {dt:.1f} s",
            "seconds": dt}


def aggregate(local_vals, dist=None, device="cpu"):
    """Combine per-rank (updates, seconds, e2e_updates, e2e_seconds): work is summed over
    ranks, time is the maximum over ranks (weak scaling, independent realisations)."""
    import torch
    v = [float(x) for x in local_vals]
    if dist is None:
        return v[0], v[1], v[2], v[3]
    t = torch.tensor(v, dtype=torch.float64, device=device)
    sums = t.clone()
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    maxs = t.clone()
    dist.all_reduce(maxs, op=dist.ReduceOp.MAX)
    return float(sums[0]), float(maxs[1]), float(sums[2]), float(maxs[3])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    res = []
    for _ in range(args.steps):
        res.append(cpu_baseline(args.workload, budget_s=max(3.0, 60.0 / max(1, args.steps))))
    value = statistics.median(r["value"] for r in res)
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "tol": 1e-8},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": res[0]["cores"],
                             "kind": "oracle", "sample": res[0]["sample"]},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_1808_07554_gb300 as pkg
    from paper_1808_07554_gb300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(build.LIB):
        build.build()
    if dist is not None:
        dist.barrier()
    pkg.load_library()

    prob = make_problem(args.workload, rank)
    nodes = prob.nx * prob.ny
    stream = torch.cuda.current_stream()
    t_setup = time.perf_counter()
    coarse_log = []
    if not args.cold_start:
        P0 = coarse_initial_pressure(prob, pkg, log=coarse_log)
        if P0 is not None:
            prob.P0 = P0
    solver = pkg.Solver.from_problem(prob, tol=args.tol, check_every=args.check_every,
                                     max_sub_iters=args.max_sub_iters, fuse_sweeps=args.fuse_sweeps,
                                     sweep_kernel=args.sweep_kernel,
                                     storage=1 if args.storage == "fp16" else 0,
                                     warm_start=1 if args.warm_start == "extrapolate" else 0)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    init_sweeps = solver.init_stats.sub_iters
    solver.set_timing(True)
    sweep_cfg = solver.sweep_config()
    fform = solver.fused_form()

    # problems with time-dependent sources get them uploaded every step (host buffers)
    def upload(n):
        if prob.sources_at is not None:
            solver.set_sources(*prob.sources_at(n * prob.dt))

    step_no = 0
    for _ in range(args.warmup):
        step_no += 1
        upload(step_no)
        solver.step(1)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    launches0, sweeps0 = solver.counters()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark_start()
    wall0 = time.perf_counter()
    step_ms, sweep_ms, ksub, statuses = [], [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        step_no += 1
        upload(step_no)
        ev0.record(stream)
        st, stats = solver.step(1)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        sweep_ms.append(stats[0].sweep_ms)
        ksub.append(stats[0].sub_iters)
        statuses.append(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks.mark_end()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    launches1, sweeps1 = solver.counters()
    gpu_launches = launches1 - launches0

    # end to end: the public API with host buffers (per step: the step's source upload when
    # the problem has one, the step, and the P and S fields read back to host memory)
    e2e_steps = max(1, min(args.steps, 5))
    h2d = 0 if prob.sources_at is None else 2 * 8 * nodes
    d2h = 2 * 4 * nodes
    # the step's result is read into page-locked host buffers (allocated once, outside)
    host_out = tuple(torch.empty((prob.ny, prob.nx), dtype=torch.float32,
                                 pin_memory=True).numpy() for _ in range(2))
    torch.cuda.synchronize()
    e2e_updates = 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_no += 1
        upload(step_no)
        st, stats = solver.step(1)
        solver.fields(out=host_out)
        e2e_updates += nodes * (stats[0].sub_iters + 1)
    e2e_s = time.perf_counter() - t0
    solver.close()

    total_ms = float(np.sum(step_ms))
    updates = nodes * (int(np.sum(ksub)) + args.steps)
    updates_all, time_max, e2e_all, e2e_max = aggregate(
        [updates, total_ms / 1e3, e2e_updates, e2e_s], dist, device="cuda")
    if rank != 0:
        return 0

    peak, peak_kind = peaks()
    sweeps_timed = int(np.sum(ksub))
    avg_sweep_s = float(np.sum(sweep_ms)) / 1e3 / max(1, sweeps_timed)
    fused = sweep_cfg[0]
    avg_launch_s = avg_sweep_s * fused
    bpn = BYTES_PER_SWEEP_NODE_FP16 if args.storage == "fp16" else BYTES_PER_SWEEP_NODE
    achieved = bpn * nodes / avg_launch_s / 1e9
    # the captured traffic belongs to one FP32 launch form; any other choice of the
    # autotuner has no capture here
    form = ((args.workload, FUSED_FORM_NAMES.get(fform, "?"), sweep_cfg[2]) if fused > 1
            else (args.workload, "single", sweep_cfg[1]))
    traffic = NCU_TRAFFIC_PER_LAUNCH.get(form) if args.storage == "fp32" else None
    line = {
        "metric": "MLUPS", "value": updates_all / time_max / 1e6, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.storage == "fp32" else "f16 storage, f32 arithmetic",
        "data": "synthetic",
        "config": {"workload": args.workload, "nx": prob.nx, "ny": prob.ny, "tol": args.tol,
                   "storage": args.storage, "warm_start": args.warm_start,
                   "check_every": args.check_every, "fuse_sweeps": args.fuse_sweeps,
                   "sweep_kernel": sweep_cfg[1], "sweep_tile": [sweep_cfg[2], sweep_cfg[3]],
                   "fused_form": FUSED_FORM_NAMES.get(fform, "none"),
                   "l2": "flushed before every timed step",
                   "sub_iters_per_step": ksub, "statuses": statuses,
                   "init_sweeps": init_sweeps, "setup_s": round(setup_s, 2),
                   "coarse_levels": coarse_log,
                   "initial_guess": "P0 = 0" if args.cold_start or prob.wells == [] else
                                    "P0 from the same problem on a 4x coarser lattice (set-up)",
                   "wall_s": round(wall, 3),
                   "parallelism": f"{world} independent realisations (seed 2 + rank)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": ("pressure sweep (fused stream + collide, Eq. 3-1), "
                                + (("FP16 populations, " + SWEEP_KERNEL_NAMES.get(sweep_cfg[1], "?"))
                                   if args.storage == "fp16"
                                   else ((f"{fused} sweeps per launch "
                                          + FUSED_FORM_TEXT.get(fform, "?"))
                                         if fused > 1 else
                                         SWEEP_KERNEL_NAMES.get(sweep_cfg[1], "?"))
                                   + (", autotuned" if args.sweep_kernel == 0 else ""))),
                     "bytes_per_launch": bpn * nodes, "sweeps_per_launch": fused,
                     "avg_launch_us": avg_launch_s * 1e6,
                     # a launch of several sweeps moves one sweep's bytes: its sweeps at the
                     # single-sweep byte count, for comparison with one-sweep kernels
                     "sweep_equivalent_gbs": fused * achieved,
                     "launch_time_includes": ("the residual finalize kernel of every "
                                              f"{args.check_every}th sweep"),
                     "peak_kind": peak_kind},
        "e2e": {"value": e2e_all / e2e_max / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(gpu_launches),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline(args.workload).items()
                                if k != "seconds"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# bytes per node of the once-per-step kernels: S refresh 44, saturation update 124, rebase 76
BYTES_PER_STEP_NODE = 244


def run_batch(args):
    """Batched realisations: every member created (and its t = 0 pressure solved) alone,
    then all advanced by one lbm2p_batch per step; afterwards the same members stepped one
    after another through their own handles, for comparison."""
    import torch
    import paper_1808_07554_gb300 as pkg
    from paper_1808_07554_gb300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(build.LIB):
        build.build()
    if dist is not None:
        dist.barrier()
    pkg.load_library()

    probs = batch_members(args.workload, rank)
    nodes = np.array([p.nx * p.ny for p in probs], dtype=np.int64)
    stream = torch.cuda.current_stream()
    t_setup = time.perf_counter()
    solvers, init_sweeps = [], 0
    for p in probs:
        if not args.cold_start:
            P0 = coarse_initial_pressure(p, pkg)
            if P0 is not None:
                p.P0 = P0
        s = pkg.Solver.from_problem(p, tol=1e-8, check_every=args.check_every,
                                    max_sub_iters=args.max_sub_iters,
                                    sweep_kernel=args.sweep_kernel,
                                    warm_start=1 if args.warm_start == "extrapolate" else 0)
        init_sweeps += s.init_stats.sub_iters
        solvers.append(s)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    batch = pkg.Batch(solvers)
    for _ in range(args.warmup):
        batch.step(1)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    launches0, tiles = batch.counters()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark_start()
    step_ms, kmat, statuses = [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev0.record(stream)
        st, stats = batch.step(1)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        kmat.append([x.sub_iters for x in stats[0]])
        statuses.append(st)
    torch.cuda.synchronize()
    clocks.mark_end()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    gpu_launches = batch.counters()[0] - launches0
    k = np.array(kmat, dtype=np.int64)                       # [steps, members]
    updates = int(np.sum(k * nodes[None, :]) + args.steps * nodes.sum())
    step_bytes = float(np.sum((BYTES_PER_SWEEP_NODE * k + BYTES_PER_STEP_NODE) * nodes[None, :]))
    total_ms = float(np.sum(step_ms))

    # end to end: batch step + P and S of every member read back to host memory
    e2e_steps = max(1, min(args.steps, 3))
    e2e_updates = 0
    # page-locked host buffers for every member's P and S (allocated once, outside)
    host_out = [tuple(torch.empty((s.ny, s.nx), dtype=torch.float32, pin_memory=True).numpy()
                      for _ in range(2)) for s in solvers]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st, stats = batch.step(1)
        for s, out in zip(solvers, host_out):
            s.fields(out=out)
        e2e_updates += int(sum((x.sub_iters + 1) * n for x, n in zip(stats[0], nodes)))
    e2e_s = time.perf_counter() - t0
    batch.close()

    # the same members one after another (each its own graph-resident step)
    seq_steps = max(1, min(args.steps, 3))
    seq_updates = 0
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(seq_steps):
        for s, n in zip(solvers, nodes):
            st, stats = s.step(1)
            seq_updates += int(n) * (stats[0].sub_iters + 1)
    ev1.record(stream)
    ev1.synchronize()
    seq_s = ev0.elapsed_time(ev1) / 1e3
    for s in solvers:
        s.close()

    updates_all, time_max, e2e_all, e2e_max = aggregate(
        [updates, total_ms / 1e3, e2e_updates, e2e_s], dist, device="cuda")
    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    achieved = step_bytes / (total_ms / 1e3) / 1e9
    sizes = {int(n): int(c) for n, c in zip(*np.unique([p.nx for p in probs], return_counts=True))}
    line = {
        "metric": "MLUPS", "value": updates_all / time_max / 1e6, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "members": len(probs),
                   "sizes": {f"{n}x{n}": c for n, c in sizes.items()},
                   "nodes": int(nodes.sum()), "tol": 1e-8, "check_every": args.check_every,
                   "warm_start": args.warm_start,
                   "l2": "flushed before every timed step",
                   "sub_iters_max_per_step": [int(x) for x in k.max(axis=1)],
                   "sub_iters_mean_per_step": [round(float(x), 1) for x in k.mean(axis=1)],
                   "statuses": statuses, "init_sweeps_total": int(init_sweeps),
                   "setup_s": round(setup_s, 2), "tiles_per_batched_sweep": int(tiles),
                   "one_at_a_time_mlups": seq_updates / seq_s / 1e6,
                   "one_at_a_time_steps": seq_steps,
                   "parallelism": f"{world} x {len(probs)} independent realisations"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": None,
                     "kernel": "whole batched step (kb_sweep dominant): algorithmic bytes of "
                               "every kernel / step time",
                     "bytes_per_step": step_bytes / args.steps, "peak_kind": peak_kind},
        "e2e": {"value": e2e_all / e2e_max / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(8 * nodes.sum())},
        "gpu_launches": int(gpu_launches),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k2: v for k2, v in cpu_baseline(args.workload).items()
                                if k2 != "seconds"}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="five_spot_1024")
    ap.add_argument("--check-every", type=int, default=None,
                    help="sweeps between residual checks (default: 16 for solves that continue "
                         "from the previous step, 8 with the warm start, whose steps take 16-24 "
                         "sweeps)")
    ap.add_argument("--max-sub-iters", type=int, default=10_000_000)
    ap.add_argument("--cold-start", action="store_true",
                    help="start the t = 0 pressure solve from P0 = 0 instead of a coarse solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fuse-sweeps", type=int, default=0, choices=[0, 1, 2, 4],
                    help="pressure sweeps per launch: 0 = autotuned, 1, 2 or 4")
    ap.add_argument("--warm-start", choices=["none", "extrapolate"], default="none",
                    help="start of each pressure solve: the previous step's populations (none) "
                         "or their equilibrium part moved to 2 P^n - P^(n-1) (extrapolate)")
    ap.add_argument("--storage", choices=["fp32", "fp16"], default="fp32",
                    help="pressure populations during the sub-iteration: FP32 or FP16 deviations")
    ap.add_argument("--tol", type=float, default=1e-8,
                    help="relative increment that ends a pressure solve")
    ap.add_argument("--sweep-kernel", type=int, default=0, choices=[0, 1, 2, 3],
                    help="single-sweep kernel: 0 = autotuned, 1 = float4, 2 = one node per "
                         "thread, 3 = staged rows")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.check_every is None:
        # a check period has a fixed cost (the checking launch, the finalize kernel and the
        # graph's loop condition): at 1024^2 about 12 us, 10 % of eight sweeps; checking every
        # 16 sweeps halves it for 0.7 % more sweeps per converged step
        args.check_every = 8 if args.warm_start == "extrapolate" else 16
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload]["kind"] == "batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the two-phase Darcy LB solver (one JSON line on stdout).

Workload (default): the quarter five-spot of 4096 x 4096 nodes (ln K a seeded Gaussian
random field, sigma 1, correlation length 16 cells; no-flux walls; injector and producer
of rate 1e-3 at opposite corners; S0 = 0.2; phi = 0.2, beta = 0.4, mu_w = 1, mu_n = 2,
D_s = 0.01, tau_p = 1, tau_s = 0.8), FP32 populations, each physical step sub-iterating the
pressure to a relative increment of 1e-8.  A step = S refresh + pressure sub-iteration +
saturation update.  The t = 0 initialisation (the pressure solve, started from the same
problem solved on a 4x coarser lattice unless --cold-start) is set-up, outside the timing;
its solve is timed on the device on its own and reported beside the line.

Metric: MLUPS = nodes x (pressure sweeps + 1 saturation update) / time, summed over the
timed steps (and over ranks).  L2 is flushed before every timed step; each step is timed
with CUDA events on the solver's stream.

Roofline of the dominant kernel (the pressure sweep launch): algorithmic bytes = 68 B per
node and pressure sweep (8 populations read and written, plus 1/tau_f) x the sweeps one
launch performs x nodes, over the launch's average device time (CUDA events around the
sweep batches, on the solver's stream), against the measured HBM copy bandwidth.  A launch
that carries two sweeps moves the populations once, so this fraction can exceed 1; the
DRAM bytes such a launch really moves (from an ncu capture of the same kernel source) give
the DRAM-actual fraction beside it.

Workload batch_five_spot_64: 64 independent five-spot realisations with sizes drawn from
{128, 256, 512}^2 (sigma, correlation length and viscosity ratio drawn per member), advanced
together by one lbm2p_batch per step; the line also reports the same members stepped one
after another.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload five_spot_4096|five_spot_1024|manufactured_64|batch_five_spot_64|
                                batch_five_spot_mixed]
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
from paper_1808_07554_gb300.initial_guess import coarse_initial_pressure  # noqa: E402

# algorithmic bytes per node and pressure sweep (the paper's form of the sweep): 8
# populations read and written + 1/tau_f; f_0 is never needed, the sparse wells add nothing
BYTES_PER_NODE_SWEEP = 68
# bytes per node the FP32 deviation storage really moves per launch (one pass over the
# populations whatever the sweeps per launch): the 68 above + the reference pressure R
BYTES_MOVED_PER_NODE = 72
# with FP16 storage: 8 populations x (2 + 2) B + the node pressure read and written + 1/tau_f
BYTES_PER_SWEEP_NODE_FP16 = 44
WORKLOADS = {
    "five_spot_4096": dict(kind="five_spot", n=4096),
    "five_spot_1024": dict(kind="five_spot", n=1024),
    # larger than L2 but a fraction of the 4096^2 footprint: the size of the ncu captures
    "five_spot_2048": dict(kind="five_spot", n=2048),
    "manufactured_64": dict(kind="manufactured", n=64),
    # independent five-spot realisations of uneven sizes advanced by one batch (lbm2p_batch)
    "batch_five_spot_64": dict(kind="batch", count=64, sizes=(128, 256, 512)),
    # the batched workload's full size set, 1024^2 members included (64 realisations)
    "batch_five_spot_mixed": dict(kind="batch", count=64, sizes=(128, 256, 512, 1024)),
}
DEFAULT_WORKLOAD = "five_spot_4096"
SWEEP_KERNEL_NAMES = {1: "four nodes per thread (128-bit accesses)", 2: "one node per thread",
                      3: "rows staged in shared memory by bulk async copies"}
# CUDA sources each launch form is compiled from; their hash keys the ncu captures below
KERNEL_SOURCES = {
    "two_sweep": ["sweep_rows.cu", "lbm2p_node.cuh", "lbm2p_device.cuh", "lbm2p_async.cuh"],
    "single": ["kernels.cu", "sweep_rows.cu", "lbm2p_node.cuh", "lbm2p_device.cuh",
               "lbm2p_async.cuh"],
}
# DRAM bytes per pressure-sweep launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture, keyed by workload and launch form (sweeps per launch, fused form, tile
# width); each entry carries the hash of the kernel sources it was taken from and the
# summary under profiles/ that holds the command.  A capture whose hash differs from the
# sources being run is stale and is not reported.
NCU_TRAFFIC_PER_LAUNCH = {
    # k_pressure_rows2<0, 4, 6, 7> (4 consumer warps, 6 slots, 16 rows, seven-block register
    # cap), mean of 3 launches: 734.4 + 494.7, 738.9 + 495.4, 734.4 + 491.8 MB
    ("five_spot_4096", "staged_rows", 120): {
        "bytes": 1229841323, "sources": "a38cf4db413179c4",
        "profile": "profiles/pressure_sweeps_fused_rows_five_spot_4096.md"},
}
FUSED_FORM_NAMES = {1: "stages", 2: "staged_rows", 3: "direct"}
FUSED_FORM_TEXT = {1: "on shared-memory stages", 2: "on rows staged by bulk copies",
                   3: "with direct loads"}


def log(msg: str) -> None:
    """Progress of the set-up and of long phases, on stderr (the JSON line stays alone on
    stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def kernel_source_hash(form: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[form]:
        with open(os.path.join(ROOT, "paper_1808_07554_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(form, src_hash: str):
    """(DRAM bytes per launch, profile summary) captured by ncu for this launch form, or
    (None, None) when there is no capture or the kernel sources changed since it was taken."""
    cap = NCU_TRAFFIC_PER_LAUNCH.get(form)
    if cap is None or cap["sources"] != src_hash:
        return None, None
    return cap["bytes"], cap["profile"]


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


def train_operator(pkg, args):
    """Set-up of --warm-start learned: quarter five-spot realisations at the training size
    (GRF ln K with sigma 1 and correlation length 16 cells, seeds 6000 + r) stepped by the
    solver, their converged fields recorded, and the five-layer operator trained on them."""
    import torch
    from paper_1808_07554_gb300.operator import PressureOperator, record_snapshots, train
    t0 = time.perf_counter()
    probs = [W.quarter_five_spot(args.op_size, seed=6000 + r) for r in range(args.op_realisations)]
    gen_log = []
    runs = record_snapshots(pkg, probs, args.op_steps, log=gen_log)
    t1 = time.perf_counter()
    op = PressureOperator(seed=1)
    train_log = []
    losses = train(op, runs, epochs=args.op_epochs, batch=16, lr=1e-3,
                   max_seconds=args.op_seconds, log=train_log)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del runs
    snaps = args.op_realisations * (args.op_steps - 1)
    return op, {"training_size": args.op_size, "realisations": args.op_realisations,
                "steps_each": args.op_steps, "snapshots": snaps,
                "data_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1),
                "epochs": train_log, "final_loss": losses[-1] if losses else None,
                "sweeps_in_data": int(sum(g["sweeps"] for g in gen_log))}


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
# sweeps per sample step of the oracle: (all host cores, one thread); fixed counts, so that
# every run times the same work (a step = S refresh + the sweeps + the saturation update)
CPU_SAMPLE_SWEEPS = {"five_spot_4096": (48, 4), "five_spot_1024": (400, 40),
                     "manufactured_64": (4000, 2000), "batch_five_spot_64": (400, 40),
                     "batch_five_spot_mixed": (400, 40)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), with the machine type."""
    import platform
    name = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        fields = {ln.split(":", 1)[0].strip(): ln.split(":", 1)[1].strip()
                  for ln in out.splitlines() if ":" in ln}
        name = fields.get("Model name") or fields.get("Vendor ID") or ""
    except Exception:
        pass
    if not name:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return f"{name or 'unknown'} ({platform.machine()})"


def oracle_sample(orc, nodes: int, sweeps: int):
    """One physical step of the oracle with a replayed sweep count: (lattice updates, s)."""
    t0 = time.perf_counter()
    orc.step(1, replay=[sweeps])
    return nodes * (sweeps + 1), time.perf_counter() - t0


def cpu_baseline(name: str, reps: int = 3):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the workload:
    `reps` steps of a fixed sweep count on all cores (median), and fewer sweeps on one thread."""
    import oracle as O
    prob = make_problem(name)
    orc = O.Oracle(prob, tol=1e-8, init_replay=0)
    nodes = prob.nx * prob.ny
    sw_all, sw_one = CPU_SAMPLE_SWEEPS.get(name, (100, 10))
    cores = O.set_threads(os.cpu_count() or 1)
    runs = [oracle_sample(orc, nodes, sw_all) for _ in range(reps)]
    all_rates = sorted(u / t / 1e6 for u, t in runs)
    O.set_threads(1)
    u1, t1 = oracle_sample(orc, nodes, sw_one)
    O.set_threads(cores)
    orc.close()
    value = all_rates[len(all_rates) // 2]
    return {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": (f"{name}: {reps} physical steps of {sw_all} pressure sweeps + 1 "
                       f"saturation update on the {prob.nx}x{prob.ny} lattice, all "
                       f"{cores} host threads ({sum(t for _, t in runs):.1f} s; median); one "
                       f"thread: 1 step of {sw_one} sweeps ({t1:.1f} s)"),
            "single_thread": {"value": u1 / t1 / 1e6, "unit": "MLUPS", "cores": 1},
            "all_cores_runs": [round(x, 2) for x in all_rates],
            "cpu_model": cpu_model(),
            "seconds": sum(t for _, t in runs) + t1}


def cpu_full_run(steps: int = 500):
    """The whole small configuration on the host: the oracle runs the 64 x 64 manufactured
    problem for `steps` physical steps, every pressure solve to r <= 1e-8, on all host threads
    and on one (minutes of CPU time: opt-in, not part of the bounded baseline)."""
    import oracle as O
    out = {"workload": "manufactured_64", "steps": steps, "cpu_model": cpu_model()}
    for label, threads in (("all_cores", os.cpu_count() or 1), ("single_thread", 1)):
        prob = make_problem("manufactured_64")
        n = O.set_threads(threads)
        orc = O.Oracle(prob, tol=1e-8)
        t0 = time.perf_counter()
        st, k, r = orc.step(steps)
        dt = time.perf_counter() - t0
        orc.close()
        out[label] = {"threads": n, "seconds": round(dt, 2), "status": int(st),
                      "sweeps": int(np.sum(k)),
                      "MLUPS": float((np.sum(k) + steps) * prob.nx * prob.ny / dt / 1e6),
                      "ms_per_step": dt / steps * 1e3}
    O.set_threads(os.cpu_count() or 1)
    return out


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
    """The oracle as it stands, on the machine's host cores: every warm-up and timed step is
    one sample of the workload (one physical step with the same fixed sweep count as the
    CPU baseline's all-core leg); the value is the median over the timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    prob = make_problem(args.workload)
    nodes = prob.nx * prob.ny
    orc = O.Oracle(prob, tol=1e-8, init_replay=0)
    cores = O.set_threads(os.cpu_count() or 1)
    sweeps = CPU_SAMPLE_SWEEPS.get(args.workload, (100, 10))[0]
    for _ in range(args.warmup):
        oracle_sample(orc, nodes, sweeps)
    runs = [oracle_sample(orc, nodes, sweeps) for _ in range(args.steps)]
    orc.close()
    rates = sorted(u / t / 1e6 for u, t in runs)
    value = rates[len(rates) // 2]
    total = sum(t for _, t in runs)
    line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / max(1, args.steps),
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nx": prob.nx, "ny": prob.ny, "tol": 1e-8},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": (f"{args.workload}: each step one physical step of "
                                        f"{sweeps} pressure sweeps + 1 saturation update on "
                                        f"the {prob.nx}x{prob.ny} lattice, {cores} host "
                                        f"threads; median of {args.steps} ({total:.1f} s)"),
                             "cpu_model": cpu_model()},
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
    torch.cuda.synchronize()
    coarse_s = time.perf_counter() - t_setup
    op_log = None
    if args.warm_start == "learned":
        op, op_log = train_operator(pkg, args)
    t_create = time.perf_counter()
    solver = pkg.Solver.from_problem(prob, tol=args.tol, check_every=args.check_every,
                                     max_sub_iters=args.max_sub_iters, fuse_sweeps=args.fuse_sweeps,
                                     sweep_kernel=args.sweep_kernel,
                                     storage=1 if args.storage == "fp16" else 0,
                                     warm_start=1 if args.warm_start == "extrapolate" else 0)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t_create
    if args.fused_shape:
        # a two-sweep launch shape pinned for the steps (the t = 0 solve ran the tuned one)
        form, warps, slots, rows = (int(v) for v in args.fused_shape.split(","))
        solver.set_fused_shape(form, warps, slots, rows)
    do_step = lambda: solver.step(1)          # noqa: E731
    if args.warm_start == "learned":
        from paper_1808_07554_gb300.operator import LearnedWarmStart
        lw = LearnedWarmStart(op, solver, np.log(prob.K))
        for _ in range(2):                     # the features need two time levels
            solver.step(1)
            lw.prime()
        do_step = lw.step
    setup_s = time.perf_counter() - t_setup
    init_sweeps = solver.init_stats.sub_iters
    # the t = 0 solve alone (device time, CUDA events inside create around the solve)
    init_solve_s = solver.init_stats.step_ms / 1e3 if solver.init_stats.step_ms >= 0 else None
    solver.set_timing(True)
    sweep_cfg = solver.sweep_config()
    fform = solver.fused_form()
    # the autotuner's candidates (us per sweep in the solve loop), fastest first
    report = sorted(solver.autotune_report(), key=lambda r: r[-1])
    autotune_best = [" ".join(str(v) for v in r) for r in report[:8]]

    # problems with time-dependent sources get them uploaded every step (host buffers)
    def upload(n):
        if prob.sources_at is not None:
            solver.set_sources(*prob.sources_at(n * prob.dt))

    step_no = 0
    for _ in range(args.warmup):
        step_no += 1
        upload(step_no)
        do_step()
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
        st, stats = do_step()
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
    # the problem has one, the step, and the P and S fields read back to host memory), over
    # as many steps as the timed region
    e2e_steps = max(1, args.steps)
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
        st, stats = do_step()
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
    fp16 = args.storage == "fp16"
    # algorithmic bytes per launch: 68 B per node and sweep x the sweeps of one launch
    bpn = BYTES_PER_SWEEP_NODE_FP16 if fp16 else BYTES_PER_NODE_SWEEP * fused
    achieved = bpn * nodes / avg_launch_s / 1e9
    form = ((args.workload, FUSED_FORM_NAMES.get(fform, "?"), sweep_cfg[2]) if fused > 1
            else (args.workload, "single", sweep_cfg[1]))
    src_form = "two_sweep" if fused > 1 else "single"
    src_hash = kernel_source_hash(src_form)
    traffic, traffic_profile = captured_traffic(form, src_hash) if not fp16 else (None, None)
    hist = {}
    for k in ksub:
        hist[str(k)] = hist.get(str(k), 0) + 1
    kernel_text = ("pressure sweep (fused stream + collide, Eq. 3-1), "
                   + (("FP16 populations, " + SWEEP_KERNEL_NAMES.get(sweep_cfg[1], "?"))
                      if fp16 else
                      ((f"{fused} sweeps per launch " + FUSED_FORM_TEXT.get(fform, "?"))
                       if fused > 1 else SWEEP_KERNEL_NAMES.get(sweep_cfg[1], "?"))
                      + (", autotuned" if args.sweep_kernel == 0 else "")))
    line = {
        "metric": "MLUPS", "value": updates_all / time_max / 1e6, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16 storage, f32 arithmetic" if fp16 else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "nx": prob.nx, "ny": prob.ny, "tol": args.tol,
                   "storage": args.storage, "warm_start": args.warm_start,
                   "check_every": args.check_every, "fuse_sweeps": args.fuse_sweeps,
                   "sweep_kernel": sweep_cfg[1], "sweep_tile": [sweep_cfg[2], sweep_cfg[3]],
                   "fused_form": FUSED_FORM_NAMES.get(fform, "none"),
                   "fused_shape_pinned": args.fused_shape,
                   "autotune_best": autotune_best,
                   "l2": "flushed before every timed step (256 MB write)",
                   "sub_iters_per_step": ksub, "sub_iters_histogram": hist,
                   "statuses": statuses,
                   "setup": {"coarse_guess_s": round(coarse_s, 2), "coarse_levels": coarse_log,
                             "create_s": round(create_s, 2),
                             "init_solve_sweeps": init_sweeps,
                             "init_solve_s": (round(init_solve_s, 3)
                                              if init_solve_s is not None else None),
                             "init_solve_from": ("P0 = 0" if args.cold_start or prob.wells == []
                                                 else "P0 from the same problem on a 4x "
                                                      "coarser lattice"),
                             "total_s": round(setup_s, 2),
                             "note": ("create_s = kernel autotuning + uploads + the t = 0 "
                                      "solve; init_solve_s is that solve alone")},
                   "wall_s": round(wall, 3),
                   "learned_operator": op_log,
                   "parallelism": f"{world} independent realisations (seed 2 + rank)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kernel_text,
                     "bytes_per_launch": bpn * nodes,
                     "bytes_model": ("44 B per node and sweep (FP16 storage)" if fp16 else
                                     f"68 B per node and sweep x {fused} sweeps per launch"),
                     "sweeps_per_launch": fused,
                     "avg_launch_us": avg_launch_s * 1e6,
                     "launch_time_includes": ("the residual finalize kernel of every "
                                              f"{args.check_every}th sweep"),
                     "dram_bytes_moved_model": (None if fp16 else BYTES_MOVED_PER_NODE * nodes),
                     "dram_frac": (traffic / avg_launch_s / 1e9 / peak
                                   if traffic is not None else None),
                     "traffic_source": (f"ncu capture, {traffic_profile}" if traffic is not None
                                        else "no ncu capture of these kernel sources"),
                     "kernel_sources": src_hash,
                     "peak_kind": peak_kind},
        "e2e": {"value": e2e_all / e2e_max / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                "note": ("the five-spot has no per-step inputs (its wells are fixed at create)"
                         if h2d == 0 else "per-step dense sources uploaded from host memory")},
        "gpu_launches": int(gpu_launches),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cpu = {k: v for k, v in cpu_baseline(args.workload).items() if k != "seconds"}
        # the oracle's time per step at this run's own sweep counts, from its sampled rate
        # (extrapolated: the oracle is not run to convergence on the full lattice)
        upd = float(np.mean((np.asarray(ksub) + 1) * nodes))
        cpu["ms_per_step_extrapolated"] = upd / (cpu["value"] * 1e6) * 1e3
        cpu["ms_per_step_extrapolated_single_thread"] = (
            upd / (cpu["single_thread"]["value"] * 1e6) * 1e3)
        line["cpu_baseline"] = cpu
    if args.cpu_full_run and rank == 0:
        line["cpu_full_run"] = cpu_full_run()
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
    for i, p in enumerate(probs):
        t_m = time.perf_counter()
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
        log(f"member {i}: {p.nx}x{p.ny}, t = 0 solve {s.init_stats.sub_iters} sweeps, "
            f"{time.perf_counter() - t_m:.1f} s")
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    batch = pkg.Batch(solvers)
    for w in range(args.warmup):
        t_w = time.perf_counter()
        st, stats = batch.step(1)
        log(f"warm-up step {w}: {time.perf_counter() - t_w:.2f} s, status {st}, "
            f"sweeps max {max(x.sub_iters for x in stats[0])}")
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
    step_bytes = float(np.sum((BYTES_MOVED_PER_NODE * k + BYTES_PER_STEP_NODE) * nodes[None, :]))
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

    log(f"batched steps done: {total_ms / 1e3:.2f} s device time, e2e {e2e_s:.2f} s")
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
    log(f"one member at a time: {seq_steps} steps in {seq_s:.2f} s")
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
                     "kernel": "whole batched step (kb_sweep for the small members, "
                               "k_pair_batch, two sweeps per launch, for those of 512^2 and "
                               "up): 72 B per node and sweep + the per-step kernels' bytes / "
                               "step time",
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--check-every", type=int, default=None,
                    help="sweeps between residual checks (default: 16 for solves that continue "
                         "from the previous step, 8 with the warm start, whose steps take 16-24 "
                         "sweeps)")
    ap.add_argument("--max-sub-iters", type=int, default=10_000_000)
    ap.add_argument("--cold-start", action="store_true",
                    help="start the t = 0 pressure solve from P0 = 0 instead of a coarse solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full-run", action="store_true",
                    help="also run the 64 x 64 manufactured configuration's 500 steps with the "
                         "oracle on the host (minutes)")
    ap.add_argument("--fuse-sweeps", type=int, default=0, choices=[0, 1, 2, 4],
                    help="pressure sweeps per launch: 0 = autotuned, 1, 2 or 4")
    ap.add_argument("--warm-start", choices=["none", "extrapolate", "learned"], default="none",
                    help="start of each pressure solve: the previous step's populations (none), "
                         "their equilibrium part moved to 2 P^n - P^(n-1) (extrapolate) or to "
                         "the five-layer operator's prediction (learned; trained first, at set-up, "
                         "on snapshots the solver produces)")
    ap.add_argument("--op-size", type=int, default=256, help="training lattice size (learned)")
    ap.add_argument("--op-realisations", type=int, default=20)
    ap.add_argument("--op-steps", type=int, default=1001,
                    help="steps recorded per training realisation")
    ap.add_argument("--op-epochs", type=int, default=2)
    ap.add_argument("--op-seconds", type=float, default=120.0, help="cap on training time")
    ap.add_argument("--storage", choices=["fp32", "fp16"], default="fp32",
                    help="pressure populations during the sub-iteration: FP32 or FP16 deviations")
    ap.add_argument("--tol", type=float, default=1e-8,
                    help="relative increment that ends a pressure solve")
    ap.add_argument("--fused-shape", default=None,
                    help="form,warps,slots,rows: pin the two-sweep launch shape of the steps "
                         "(lbm2p_set_fused_shape; form 2 = staged rows, 3 = direct loads)")
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
        args.check_every = 16 if args.warm_start == "none" else 8
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload]["kind"] == "batch":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

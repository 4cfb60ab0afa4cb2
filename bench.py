#!/usr/bin/env python3
"""Benchmark of the WENO-ZA6 hot path on GB300.

One benchmark step = one SSP-RK3 step (three right-hand-side stages: GLF
splitting, Roe characteristic projection, WENO-ZA6 reconstruction, flux
difference, stage combination, CFL reduction) of 2D Euler on the seeded
four-quadrant workload, 2048 x 2048 cells, FP64.  The metric is cell-updates
per second (one cell advanced one full Runge-Kutta step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 restatement of the
paper) on the host cores, on a bounded window of the same workload.
Under torchrun (N > 1) every rank advances its own replica (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D Euler cell-updates/s FP64 vs FP32-recon; batched-solve p50/p99 latency"
UNIT = "cell-updates/s"
N_GRID = 2048
SEED = 3

# Algorithmic FP64 work of one 2D cell-update (one cell, one full SSP-RK3
# step), counted from the steps of the method rather than from the kernel:
# per face and direction the Roe average with R and L about 60 flops, the
# projection of 6 states and 6 fluxes on L (6 x 2 x 4 x 4 multiply-adds) 384,
# the GLF split 48, 8 WENO-ZA6 reconstructions of about 160 flops 1280, the
# back-projection 32, i.e. about 1.8k; two faces per cell and three stages,
# plus the per-cell primitives, flux difference and stage combination: about
# 11k flops per cell-update, 3.67k per cell and stage.  (The kernel executes
# fewer FP64 instructions than this count thanks to exact rewrites of the
# formulas; the executed count from ncu is reported beside it when the
# committed capture matches the current sources.)
FLOPS_PER_CELL_UPDATE = 11000.0
FLOPS_PER_CELL_STAGE = FLOPS_PER_CELL_UPDATE / 3.0
# Algorithmic HBM bytes per 2D cell-update: each stage reads its input state
# (32 B), stages 2 and 3 also read U^n, and each writes its output:
# 32 x (2 + 3 + 3) = 256 B.
BYTES_PER_CELL_UPDATE = 256.0
KERNEL_SOURCES = ["paper_2603_26272_gb300/csrc/weno_tiles.cuh",
                  "paper_2603_26272_gb300/csrc/weno_kernels.cu",
                  "paper_2603_26272_gb300/csrc/weno_device.cuh"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_record():
    """The committed ncu figures of the stage kernel (DRAM bytes and executed
    FP64 operations per launch at 2048^2), if they were taken on the current
    kernel sources; {} otherwise."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return {}
    if rec.get("kernel_hash") != kernel_hash():
        return {}
    return rec


def measured_peaks():
    """MEASURED_PEAKS.json of this machine pool (HBM copy bandwidth), if present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def fma_peaks(weno):
    """FMA throughput of this GPU measured now (weno_fma_rate): FP64 on
    full-mantissa operands, FP64 on short ones, FP32; best of 3 launches each,
    in TFLOP/s."""
    out = {}
    for kind in ("fp64", "fp64_short_mantissa", "fp32"):
        out[kind] = max(weno.fma_rate(kind, iters=4096 if kind != "fp32" else 65536)
                        for _ in range(3)) / 1e12
    return out


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.fh = None

    def start(self):
        try:
            self.fh = tempfile.TemporaryFile(mode="w+")
            cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.fh.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def precision_modes(weno, wl, torch, n=4096, steps=4, warmup=3):
    """Configuration 4: the quadrant workload at n x n, FP64 and
    FP32-reconstruction on the same GPU (device-timed SSP-RK3 steps)."""
    w = wl.quadrant_2d(n=n, seed=SEED)
    out = {"workload": "2D Euler %dx%d four-quadrant Riemann data (seed %d), SSP-RK3 CFL 0.5"
                       % (n, n, SEED)}
    U0 = torch.from_numpy(w["U"])
    stream = torch.cuda.current_stream()
    for prec in ("fp64", "fp32_recon"):
        d = weno.desc_for(w, precision=prec)
        U = U0.cuda()
        ws = weno.workspace(d)
        for _ in range(warmup):
            weno.step(d, U, ws=ws, sync=False)
        weno.sync_status(d, ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            weno.step(d, U, ws=ws, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        weno.sync_status(d, ws)
        ms = a.elapsed_time(b) / steps
        out[prec] = {"value": n * n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "steps": steps, "warmup": warmup}
        del U, ws
        torch.cuda.empty_cache()
    out["fp32_recon_speedup"] = out["fp32_recon"]["value"] / out["fp64"]["value"]
    out["error_vs_fp64_oracle"] = "profiles/fp32_recon_error_512.md"
    return out


def scheme_orders(weno, wl, torch, n=N_GRID, steps=4, warmup=3):
    """The central-upwind family at orders 4, 6, 8 and 10 (the Appendix
    schemes beside WENO-ZA6) on the same 2D workload, FP64, device-timed
    SSP-RK3 steps."""
    w = wl.quadrant_2d(n=n, seed=SEED)
    out = {"workload": "2D Euler %dx%d four-quadrant Riemann data (seed %d), SSP-RK3 CFL 0.5, "
                       "FP64" % (n, n, SEED)}
    U0 = torch.from_numpy(w["U"])
    stream = torch.cuda.current_stream()
    for order in (4, 6, 8, 10):
        d = weno.desc_for(w, order=order)
        U = U0.cuda()
        ws = weno.workspace(d)
        for _ in range(warmup):
            weno.step(d, U, ws=ws, sync=False)
        weno.sync_status(d, ws)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            weno.step(d, U, ws=ws, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        weno.sync_status(d, ws)
        ms = a.elapsed_time(b) / steps
        out["order%d" % order] = {"value": n * n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                                  "steps": steps, "warmup": warmup}
        del U, ws
        torch.cuda.empty_cache()
    return out


def configs_1d(weno, wl, torch):
    """Configurations 1 and 2, each a full solve to its final time through
    weno_solve (state resident on the GPU; wall time of the call, which
    includes its launches and its final status read)."""
    import time as _time
    out = {}
    for key, w, desc in (
            ("C1_advection_N200_T2", wl.advection_sine(n=200),
             "1D linear advection, N = 200, periodic [-1, 1], t = 2, FP64"),
            ("C2_shock_density_N1600_T1.8", wl.shock_density(n=1600),
             "1D Euler shock-density, N = 1600 on [-5, 5], t = 1.8, FP64"),
            ("C2_riemann_batch_64xN1600_T0.4", wl.riemann_batch(nbatch=64, n=1600, seed=2),
             "64 seeded 1D Euler Riemann problems, N = 1600 each, t = 0.4, FP64, one batch")):
        d = weno.desc_for(w)
        U0 = torch.from_numpy(np.ascontiguousarray(w["U"])).cuda()
        ws = weno.workspace(d)
        U = U0.clone()
        weno.solve(d, U, w["t_final"], ws=ws)  # warm-up
        U = U0.clone()
        torch.cuda.synchronize()
        t0 = _time.perf_counter()
        _, n = weno.solve(d, U, w["t_final"], ws=ws)
        el = _time.perf_counter() - t0
        cells = d.nbatch * d.nx * d.ny
        steps = int(np.max(n))
        out[key] = {"workload": desc, "steps": steps, "seconds": el,
                    "value": cells * float(np.sum(n)) / max(1, d.nbatch) / el, "unit": UNIT}
    return out


# admission budget of the engine when every solve goes through it (policy
# "engine"): admitted solves' cost per step, in 2D FP64 cells (about 2 tiles
# per SM of 16x16 cells on 152 SMs, with a margin).
WORK_BUDGET = 250e3


def serving(n_requests=64, seed=5, loads=(1.0, 1.25), mix="full", policy="two_lane",
            capacity=False, large_workers=2, bypass_s=0.0):
    """Configuration 5: a seeded Poisson stream of mixed 1D/2D, FP64/FP32-
    reconstruction solves of the configured sizes (2D sides 128..1024, 1D N
    256..16384, 100..1000 steps), n_requests of them (the configured 2000
    take about 20 minutes per pass).  The offered rate is `loads` x the
    one-at-a-time capacity, measured first on the same GPU; at each load the
    same arrivals are served one at a time (weno_solve, first come first
    served) and by the serving loop (`policy`: "two_lane" -- solves that fill
    the GPU alone one at a time on a low-priority stream, all others in the
    continuous-batching engine on a high-priority stream -- or "engine",
    every solve in the engine under a work budget)."""
    import torch
    from paper_2603_26272_gb300 import serve
    if mix == "full":
        sides, n1d, steps = (128, 192, 256, 384, 512, 768, 1024), (256, 16384), (100, 1000)
    else:
        sides, n1d, steps = (128, 192, 256), (256, 16384), (100, 300)
    reqs = serve.make_requests(n_requests, seed=seed, rate=None, sides_2d=sides, n1d=n1d,
                               steps=steps)
    serve.serve_one_at_a_time(reqs)  # calibration: service times back to back
    service = [r.result["done"] - r.result["admit"] for r in reqs]
    calib_thr = serve.summarize(reqs)["throughput_cell_updates_per_s"]
    free = torch.cuda.mem_get_info()[0]
    eng = serve.Engine(arena_bytes=int(min(8 << 30, free // 2)), max_slots=256)

    def run(rs):
        if policy == "two_lane":
            return serve.serve_two_lane(eng, rs, large_workers=large_workers, bypass_s=bypass_s)
        return serve.serve_continuous(eng, rs, steps_per_poll=2, work_budget=WORK_BUDGET)

    out = {"workload": "%d requests (of the configured 2000; the rest scaled as configured): "
                       "50%% 1D Euler Riemann (N log-uniform %d..%d), 50%% 2D quadrant (side in "
                       "%s); 50%% FP64, 50%% FP32-recon; %d..%d steps each; Poisson arrivals "
                       "(seed %d)" % (n_requests, n1d[0], n1d[1], list(sides), steps[0], steps[1],
                                      seed),
           "policy": policy,
           "large_lane_tiles": serve.full_wave_tiles() if policy == "two_lane" else None,
           "large_lane_workers": large_workers if policy == "two_lane" else None,
           "bypass_s": (None if bypass_s == float("inf") else bypass_s)
           if policy == "two_lane" else None,
           "work_budget_cell_units": WORK_BUDGET if policy == "engine" else None,
           "mean_service_s_one_at_a_time": float(np.mean(service)), "loads": []}
    for load in loads:
        rate = load / float(np.mean(service))
        gaps = np.random.default_rng(seed + 1).exponential(1.0 / rate, size=len(reqs))
        arr = np.cumsum(gaps) - gaps[0]
        for r, a in zip(reqs, arr):
            r.arrival = float(a)
            r.result = {}
        base = serve.summarize(serve.serve_one_at_a_time(reqs))
        for r in reqs:
            r.result = {}
        cont = serve.summarize(run(reqs))
        if policy == "two_lane":
            cont["large_lane_requests"] = sum(1 for r in reqs if r.result.get("lane") == "large")
        out["loads"].append({
            "offered_load_vs_one_at_a_time": load, "offered_rate_per_s": rate,
            "one_at_a_time": base, "continuous_batching": cont,
            "throughput_ratio": (cont["throughput_cell_updates_per_s"]
                                 / base["throughput_cell_updates_per_s"]),
            "p50_ratio": cont["p50_latency_s"] / base["p50_latency_s"],
            "p99_ratio": cont["p99_latency_s"] / base["p99_latency_s"]})
    if capacity:
        # every request present at t = 0, against the back-to-back
        # one-at-a-time calibration run above
        for r in reqs:
            r.arrival = 0.0
            r.result = {}
        sat = serve.summarize(run(reqs))
        out.update({"capacity_one_at_a_time_cell_updates_per_s": calib_thr,
                    "capacity_continuous_cell_updates_per_s": sat["throughput_cell_updates_per_s"],
                    "capacity_ratio": sat["throughput_cell_updates_per_s"] / calib_thr})
    eng.close()
    return out


def kernel_tour(weno, wl, torch, reps=3):
    """Each kernel family of the library a few times on its configuration's
    data, for per-kernel ncu captures (-k <kernel> -c 1): the 2D stage in
    FP64 and FP32 reconstruction (2048^2 quadrant), the 1D tile kernel (64
    Riemann problems x 1600), the 1D lane layout (shock-density N = 1600),
    the wavespeed pass, a domain-split stage (two strips) and the serving
    engine (a few small solves).  Prints one line per family."""
    from paper_2603_26272_gb300 import decomp, serve
    w = wl.quadrant_2d(n=N_GRID, seed=SEED)
    for prec in ("fp64", "fp32_recon"):
        d = weno.desc_for(w, precision=prec)
        U = torch.from_numpy(w["U"]).cuda()
        ws = weno.workspace(d)
        for _ in range(reps):
            weno.step(d, U, ws=ws, sync=False)
        weno.sync_status(d, ws)
        log("tour: 2D stage %s" % prec)
        del U, ws
    for w1 in (wl.riemann_batch(nbatch=64, n=1600, seed=2), wl.shock_density(n=1600)):
        d = weno.desc_for(w1)
        U = torch.from_numpy(np.ascontiguousarray(w1["U"])).cuda()
        ws = weno.workspace(d)
        for _ in range(reps):
            weno.step(d, U, ws=ws, sync=False)
        weno.sync_status(d, ws)
        log("tour: 1D nbatch %d" % d.nbatch)
    d = weno.desc_for(w)
    grp = decomp.StripGroup(d, 2)
    parts = grp.split(torch.from_numpy(w["U"]).cuda())
    for _ in range(reps):
        grp.step(parts)
    torch.cuda.synchronize()
    log("tour: strips")
    del parts, grp
    reqs = serve.make_requests(8, seed=7, sides_2d=(128, 192), n1d=(256, 4096), steps=(20, 40))
    eng = serve.Engine(arena_bytes=1 << 30, max_slots=16)
    serve.serve_continuous(eng, reqs, steps_per_poll=2)
    eng.close()
    log("tour: engine")


def _oracle_window(args):
    """One host process of the CPU baseline: the oracle, as it stands, on the
    window x window block of the bench workload around the quadrant corner
    (as its own problem with transmissive boundaries; the oracle's cost per
    cell does not depend on the data).  Runs `steps` SSP-RK3 steps after
    `warmup`, or, with steps = 0, as many as fit in `seconds`.  Returns
    (cell-updates, seconds)."""
    window, warmup, steps, seconds = args
    import oracle
    from paper_2603_26272_gb300 import workloads as wl
    w = wl.quadrant_2d(n=N_GRID, seed=SEED)
    c0 = N_GRID // 2 - window // 2
    U = np.ascontiguousarray(w["U"][:, :, c0:c0 + window, c0:c0 + window])
    del w
    g = oracle.make_grid(ndim=2, nx=window, ny=window, dx=1.0 / N_GRID, dy=1.0 / N_GRID)
    for _ in range(warmup):
        U = oracle.ssprk3_step(g, U, oracle.cfl_dt(g, U, 0.5))
    n = 0
    t0 = time.perf_counter()
    while True:
        U = oracle.ssprk3_step(g, U, oracle.cfl_dt(g, U, 0.5))
        n += 1
        el = time.perf_counter() - t0
        if (steps and n >= steps) or (not steps and el >= seconds):
            break
    return window * window * n, el


def oracle_on_host_cores(window=256, warmup=0, steps=0, seconds=10.0, workers=None):
    """The oracle on every host core at once: one process per core (spawn),
    each on its own copy of the window.  Returns the aggregate cell-update
    rate, the cores used and a description of the sample."""
    import multiprocessing as mproc
    workers = workers or os.cpu_count() or 1
    ctx = mproc.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_window, [(window, warmup, steps, seconds)] * workers)
    value = sum(c / t for c, t in res)
    per = sum(c for c, _ in res) / workers / (window * window)
    sample = ("%d x %d window of the 2048^2 quadrant workload (around the quadrant corner) on "
              "each of %d host cores at once (one single-threaded C++ oracle process per core), "
              "%.0f SSP-RK3 steps each, %.1f s" % (window, window, workers, per,
                                                    max(t for _, t in res)))
    return value, workers, sample, max(t for _, t in res)


def cpu_baseline(seconds, window=256):
    """The oracle, as it stands, on all host cores (a bounded sample)."""
    value, cores, sample, _ = oracle_on_host_cores(window, seconds=seconds)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}


def bench_config(n, parallelism="single GPU"):
    return {"workload": "2D Euler %dx%d four-quadrant Riemann data (seed %d, rho,p~U[0.1,1.5], "
                        "u,v~U[-1,1]), transmissive, FP64, WENO-ZA6 Ai-Z p=1, SSP-RK3 CFL 0.5"
                        % (n, n, SEED),
            "parallelism": parallelism,
            "l2": "inputs larger than L2 (state %.0f MB, working set %.0f MB)"
                  % (n * n * 32 / 1e6, 3 * n * n * 32 / 1e6)}


def job_timing(elapsed_ms, world, cells, steps, dist=None, device=None):
    """Whole-job throughput of N replicas: the slowest rank's timed region
    (all_reduce MAX over ranks) and every rank's cell-updates over it."""
    t_max = float(elapsed_ms)
    if dist is not None:
        import torch
        tt = torch.tensor([t_max], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return t_max, world * cells * steps / (t_max / 1e3)


def run_reference(args, rank):
    """The reference arm: the oracle (the plain CPU restatement of the paper;
    no reference implementation exists) on every host core, each core
    advancing its own copy of a 256 x 256 window of the bench workload by
    `--steps` SSP-RK3 steps after `--warmup`; value = the cores' summed rate."""
    if rank != 0:
        return
    window = 256
    value, cores, sample, el = oracle_on_host_cores(window, warmup=args.warmup,
                                                    steps=args.steps)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(N_GRID, parallelism="%d host cores" % cores),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-modes", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-orders", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--serving-mix", choices=["small", "full"], default="full",
                    help="full: the configured 2D sides 128-1024 and 100-1000 steps; small: 2D "
                         "sides 128-256, 100-300 steps")
    ap.add_argument("--serving-policy", choices=["two_lane", "engine"], default="two_lane")
    ap.add_argument("--kernel-tour", action="store_true",
                    help="run each kernel family a few times (for per-kernel ncu captures) and exit")
    ap.add_argument("--serving-loads", type=float, nargs="+", default=[1.0, 1.25],
                    help="offered loads, as multiples of the one-at-a-time capacity")
    ap.add_argument("--serving-large-workers", type=int, default=2)
    ap.add_argument("--serving-bypass", type=float, default=0.0,
                    help="seconds small solves may overtake the oldest large one (0: arrival "
                         "order between the lanes; inf: small solves always first)")
    ap.add_argument("--serving-capacity", action="store_true",
                    help="also serve every request at t = 0 (one more pass)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    from paper_2603_26272_gb300 import weno
    from paper_2603_26272_gb300 import workloads as wl

    torch.cuda.set_device(local)
    if args.kernel_tour:
        kernel_tour(weno, wl, torch)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    n = args.n
    w = wl.quadrant_2d(n=n, seed=SEED)
    d = weno.desc_for(w)
    U0 = torch.from_numpy(w["U"])
    U = U0.cuda()
    ws = weno.workspace(d, host=True)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        weno.step(d, U, ws=ws, sync=False)
    weno.sync_status(d, ws)

    # alpha-only launch time (the wavespeed pass that opens every step)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    weno.wavespeeds(d, U, ws=ws)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(5):
        weno.wavespeeds(d, U, ws=ws)
    ev[1].record(stream)
    torch.cuda.synchronize()
    alpha_ms = ev[0].elapsed_time(ev[1]) / 5

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid).replace("GPU-", "")
    except Exception:
        gpu_id = local
    clocks = Clocks(gpu_id)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        weno.step(d, U, ws=ws, sync=False)
    end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    elapsed_ms = start.elapsed_time(end)
    weno.sync_status(d, ws)
    cells = n * n
    t_max, value = job_timing(elapsed_ms, world, cells, args.steps, dist,
                              torch.device("cuda", local) if dist else None)
    ms_step = t_max / args.steps

    # end to end: the public host-buffer call, H2D + step + D2H per step
    H = U0.clone().pin_memory()
    weno.step_host(d, H, ws=ws)
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        weno.step_host(d, H, ws=ws)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    state_bytes = U0.numel() * 8

    stage_ms = (ms_step - alpha_ms) / 3.0
    flops = cells * FLOPS_PER_CELL_STAGE
    achieved = flops / (stage_ms / 1e3) / 1e12
    rec = ncu_record()
    traffic = rec.get("dram_bytes_per_launch_2048") if n == 2048 else None
    clocks_peak = Clocks(gpu_id)
    clocks_peak.start()
    peaks = fma_peaks(weno)
    clk_peak = clocks_peak.stop()
    fp64_peak = max(peaks["fp64"], peaks["fp64_short_mantissa"])
    hbm_gbs = measured_peaks().get("hbm_gbs")
    bytes_step = cells * BYTES_PER_CELL_UPDATE
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
        "frac": achieved / fp64_peak, "traffic": traffic,
        "kernel": "k_euler2d stage launch (one SSP-RK3 stage of the 2048^2 grid)",
        "stage_ms": stage_ms, "alpha_ms": alpha_ms, "flops_per_launch": flops,
        "flops_per_cell_stage": FLOPS_PER_CELL_STAGE,
        "peak_source": "measured in this run by weno_fma_rate: best FP64 FMA rate of this GPU "
                       "(short-mantissa chains %.3f, full-mantissa %.3f TFLOP/s; FP32 %.1f)"
                       % (peaks["fp64_short_mantissa"], peaks["fp64"], peaks["fp32"]),
        "fp64_peak_full_mantissa": peaks["fp64"],
        "frac_vs_full_mantissa_peak": achieved / peaks["fp64"],
        "fp32_peak": peaks["fp32"],
        "peak_clocks": clk_peak,
        "hbm": {"achieved_gbs": bytes_step / (ms_step / 1e3) / 1e9, "peak_gbs": hbm_gbs,
                "frac": (bytes_step / (ms_step / 1e3) / 1e9 / hbm_gbs) if hbm_gbs else None,
                "bytes_per_cell_update": BYTES_PER_CELL_UPDATE,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
    }
    fp64_ops = rec.get("fp64_flops_per_launch_2048")
    if fp64_ops and n == 2048:
        ex = fp64_ops / (stage_ms / 1e3) / 1e12
        instr = sum(rec.get("fp64_instructions_per_launch_2048", {}).values())
        roofline["executed"] = {"fp64_flops_per_launch": fp64_ops, "achieved": ex,
                                "frac": ex / fp64_peak,
                                "source": "ncu sm__sass_thread_inst_executed_op_d{fma,add,mul}"
                                          "_pred_on (fma = 2) of one launch, profiles/"}
        if instr:
            # every FP64 instruction takes one issue slot of the pipe, whatever
            # its flops: its rate against the measured FMA instruction rate
            roofline["executed"]["fp64_instructions_per_launch"] = instr
            roofline["executed"]["issue_frac"] = (instr / (stage_ms / 1e3)) / (fp64_peak * 1e12 / 2)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "stage_updates_per_s": 3 * value,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(n, "replicas" if world > 1 else "single GPU"),
        "roofline": roofline,
        "e2e": {"value": cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes},
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
    }
    if world > 1:  # the extra sections are single-GPU lines; don't hold N GPUs for them
        args.no_precision_modes = args.no_orders = args.no_serving = True
        args.no_cpu_baseline = True
    if not args.no_precision_modes:
        del U
        torch.cuda.empty_cache()
        result["precision_modes"] = precision_modes(weno, wl, torch)
        result["gpu_launches_precision_modes"] = 4 * 2 * (4 + 3)
    if not args.no_orders:
        result["configs_1d"] = configs_1d(weno, wl, torch)
        result["scheme_orders"] = scheme_orders(weno, wl, torch)
        result["gpu_launches_scheme_orders"] = 4 * 4 * (4 + 3)
    if not args.no_serving and rank == 0:
        log("serving stream ...")
        result["serving"] = serving(args.serving_requests, loads=tuple(args.serving_loads),
                                    mix=args.serving_mix,
                                    policy=args.serving_policy, capacity=args.serving_capacity,
                                    large_workers=args.serving_large_workers,
                                    bypass_s=args.serving_bypass)
    if rank == 0 and not args.no_cpu_baseline:
        log("timing the CPU oracle on the host cores ...")
        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Error of every GPU output against the FP64 oracle, for every configuration.

For each seeded workload the oracle (FP64, CPU), the GPU FP64 path and the
GPU FP32-reconstruction mode advance the same data with the oracle's CFL
steps (one common step for a batch) to the configuration's end, and the
relative L1 and L_inf error of every conserved component is printed as a
markdown table (relative L1 = sum|a - b| / sum|b|, relative L_inf =
max|a - b| / max|b|).  Where an exact solution exists (linear advection, the
Riemann problems) the oracle's own error against it is printed too.  For the
1D runs the last columns give the oracle's own spread: the same run from
the input times (1 +- 1e-16) (random signs), and the same run in the oracle
build whose final sums are added in the opposite order, each against the
stock run, and whether the FP64 GPU result meets 1e-10 and the full-run
bound max(1e-10, 4 x spread).  With p = 1 and eps = 1e-40 some runs amplify
rounding far above 1e-10; the GPU's difference is to be read against that
spread.
Not collected by pytest (a measurement: every oracle run goes to its own spawned
process first, then the GPU replays the oracle's steps); its
output is summarised in profiles/errors_by_config.md.

    python tests/report_errors.py [--n2d 512] [--steps2d 200] [--jobs N]
"""
import argparse
import multiprocessing
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import torch  # noqa: E402
from paper_2603_26272_gb300 import weno  # noqa: E402
from paper_2603_26272_gb300 import workloads as wl  # noqa: E402


def rel(a, b, k):
    x, y = a[:, k], b[:, k]
    sy = np.abs(y).sum()
    my = np.abs(y).max()
    return (np.abs(x - y).sum() / sy if sy > 0 else 0.0,
            np.abs(x - y).max() / my if my > 0 else 0.0)


def grid_kwargs(d):
    sysname = {0: "advection", 1: "euler", 2: "burgers", 3: "buckley_leverett"}[d.system]
    return dict(system=sysname, ndim=d.ndim, nbatch=d.nbatch, nx=d.nx, ny=d.ny,
                dx=(d.x1 - d.x0) / d.nx, dy=(d.y1 - d.y0) / d.ny if d.ndim == 2 else 1.0,
                bc_x={0: "transmissive", 1: "periodic"}[d.bc_x],
                bc_y={0: "transmissive", 1: "periodic"}[d.bc_y], gamma=d.gamma,
                eps=d.eps, mu0=d.mu0, p=d.p, ai=d.ai, adv_speed=d.adv_speed, order=d.order)


def oracle_job(job):
    """One oracle run (in a worker process): the workload `job["wl"]` (a
    workloads function and its arguments, so the worker rebuilds the same
    seeded data) advanced with the oracle's own CFL steps to t_final or for
    `steps` steps; kind "stock", "pert" (input times 1 +- 1e-16, random
    signs) or "rev" (the reversed-summation build).  Returns the final state
    and the steps taken."""
    fn, kw = job["wl"]
    w = getattr(wl, fn)(**kw)
    g = oracle.make_grid(**job["grid"])
    U = np.ascontiguousarray(w["U"])
    if job["kind"] == "pert":
        U = U * (1 + 1e-16 * np.random.default_rng(1).choice([-1.0, 1.0], size=U.shape))
    t_final, steps = job["t_final"], job["steps"]

    def go(U):
        t, dts = 0.0, []
        while steps is None or len(dts) < steps:
            dt = float(oracle.cfl_dt(g, U, job["cfl"]).min())
            if t_final is not None:
                if t >= t_final:
                    break
                dt = min(dt, t_final - t)
            U = oracle.ssprk3_step(g, U, dt)
            t += dt
            dts.append(dt)
        return U, dts

    if job["kind"] == "rev":
        with oracle.rounding_variant("reversed"):
            return go(U)
    return go(U)


def gpu_run(w, dts, order=6, with_fp32=True):
    """GPU FP64 (and FP32-recon) advanced with the oracle's steps."""
    d64 = weno.desc_for(w, order=order)
    d32 = weno.desc_for(w, precision="fp32_recon") if with_fp32 else None
    U0 = np.ascontiguousarray(w["U"])
    A = torch.from_numpy(U0.copy()).cuda()
    B = torch.from_numpy(U0.copy()).cuda() if with_fp32 else None
    for dt in dts:
        weno.step(d64, A, dt=dt, sync=False)
        if with_fp32:
            weno.step(d32, B, dt=dt, sync=False)
    torch.cuda.synchronize()
    return A.cpu().numpy(), (B.cpu().numpy() if with_fp32 else None)


NAMES = {1: ["u"], 3: ["rho", "rho u", "E"], 4: ["rho", "rho u", "rho v", "E"]}


def table(title, U_o, a, b, extra="", spread=None):
    """One markdown table per configuration.  With `spread` (the oracle run
    from the perturbed input and in the reversed-summation build) the
    columns give both spreads and whether the FP64 GPU result meets the
    flat 1e-10 bound and the full-run bound max(1e-10, 4 x spread)."""
    nc = U_o.shape[1]
    print("\n### %s\n" % title)
    if extra:
        print(extra + "\n")
    head = "| component | FP64 GPU rel L1 | FP64 GPU rel Linf |"
    sep = "|---|---|---|"
    if b is not None:
        head += " FP32-recon rel L1 | FP32-recon rel Linf |"
        sep += "---|---|"
    if spread is not None:
        head += (" oracle spread, input x(1+-1e-16), rel Linf | oracle spread, reversed sums, "
                 "rel Linf | meets 1e-10 | meets the full-run bound |")
        sep += "---|---|---|---|"
    else:
        head += " meets 1e-10 |"
        sep += "---|"
    print(head)
    print(sep)
    for k in range(nc):
        e1, einf = rel(a, U_o, k)
        row = "| %s | %.2e | %.2e |" % (NAMES[nc][k], e1, einf)
        if b is not None:
            row += " %.2e | %.2e |" % rel(b, U_o, k)
        if spread is not None:
            sp_p = rel(spread[1], spread[0], k)[1]
            sp_r = rel(spread[2], spread[0], k)[1]
            bound = max(1e-10, 4.0 * max(sp_p, sp_r))
            row += " %.2e | %.2e | %s | %s |" % (sp_p, sp_r, "yes" if einf <= 1e-10 else "no",
                                                  "yes" if einf <= bound else "no")
        else:
            row += " %s |" % ("yes" if einf <= 1e-10 else "no")
        print(row)
    sys.stdout.flush()


def riemann_exact_err(w, U_o, t):
    """Oracle's L1 error in density against the exact Riemann solutions."""
    errs = []
    for b in range(U_o.shape[0]):
        left, right = w["states"][b, 0], w["states"][b, 1]
        try:
            rho, _, _, _ = oracle.riemann_exact(left, right, w["x"], t, x0=float(w["x0"][b]))
        except oracle.OracleError:  # a vacuum forms: no exact solution to compare
            continue
        errs.append(np.abs(U_o[b, 0, 0] - rho).mean())
    return float(np.mean(errs)), float(np.max(errs)), len(errs)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n2d", type=int, default=512)
    ap.add_argument("--steps2d", type=int, default=200)
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1,
                    help="oracle runs in parallel (one process each, spawned)")
    args = ap.parse_args()
    t0 = time.time()
    print("# GPU outputs against the FP64 oracle, every configuration")

    # (title, workload function and arguments, order, steps, FP32 too, spread runs)
    cfgs = [("C1", ("advection_sine", {"n": 200}), 6, None, True, True),
            ("C2sd", ("shock_density", {"n": 1600}), 6, None, True, True),
            ("C2rb", ("riemann_batch", {"nbatch": 64, "n": 1600, "seed": 2}), 6, None, True, True),
            ("C3", ("quadrant_2d", {"n": args.n2d, "seed": 3}), 6, args.steps2d, True, False),
            ("burgers", ("burgers_sine", {"n": 200}), 6, None, True, True),
            ("bl", ("buckley_leverett", {}), 6, None, True, True)]
    cfgs += [("sod%d" % o, ("shock_tube", {"name": "sod", "n": 200}), o, None, False, True)
             for o in (4, 8, 10)]
    jobs, keys = [], []
    for key, spec, order, steps, _, spread in cfgs:
        w = getattr(wl, spec[0])(**spec[1])
        d = weno.desc_for(w, order=order)
        base = {"wl": spec, "grid": grid_kwargs(d), "cfl": d.cfl, "steps": steps,
                "t_final": None if steps is not None else w["t_final"]}
        for kind in (("stock", "pert", "rev") if spread else ("stock",)):
            jobs.append(dict(base, kind=kind))
            keys.append((key, kind))
    # every oracle run at once, in spawned processes (no GPU work in them)
    with multiprocessing.get_context("spawn").Pool(min(args.jobs, len(jobs))) as pool:
        res = dict(zip(keys, pool.map(oracle_job, jobs, chunksize=1)))

    def report(key, spec, order, with_fp32, title_fn, extra_fn=None):
        w = getattr(wl, spec[0])(**spec[1])
        U_o, dts = res[(key, "stock")]
        a, b = gpu_run(w, dts, order=order, with_fp32=with_fp32)
        spread = ((U_o, res[(key, "pert")][0], res[(key, "rev")][0])
                  if (key, "pert") in res else None)
        extra = extra_fn(w, U_o, a, sum(dts)) if extra_fn else ""
        table(title_fn(len(dts)), U_o, a, b, extra, spread=spread)

    def c1_extra(w, U_o, a, t):
        ex = w["exact"](w["x"], t)
        e_o = np.abs(U_o[0, 0, 0] - ex)
        return ("oracle against the exact solution: L1 (mean) %.2e, Linf %.2e; GPU FP64 against "
                "it: %.2e, %.2e" % (e_o.mean(), e_o.max(), np.abs(a[0, 0, 0] - ex).mean(),
                                    np.abs(a[0, 0, 0] - ex).max()))

    def rb_extra(w, U_o, a, t):
        m, mx, cnt = riemann_exact_err(w, U_o, t)
        return ("oracle density against the exact Riemann solutions (%d problems without "
                "vacuum): mean L1 %.2e, worst problem %.2e" % (cnt, m, mx))

    spec = dict((c[0], c) for c in cfgs)
    report("C1", spec["C1"][1], 6, True,
           lambda n: "C1 linear advection, N = 200, periodic [-1, 1], t = 2 (%d steps)" % n, c1_extra)
    report("C2sd", spec["C2sd"][1], 6, True,
           lambda n: "C2 1D Euler shock-density, N = 1600 on [-5, 5], t = 1.8 (%d steps)" % n)
    report("C2rb", spec["C2rb"][1], 6, True,
           lambda n: "C2 batch of 64 random Riemann problems, N = 1600, t = 0.4 (%d common steps)"
           % n, rb_extra)
    report("C3", spec["C3"][1], 6, True,
           lambda n: "C3 / C4 2D quadrant (seed 3) at %d^2, %d steps" % (args.n2d, n))
    report("burgers", spec["burgers"][1], 6, True,
           lambda n: "Burgers (Section 4.1), N = 200, t = 0.2 (%d steps)" % n)
    report("bl", spec["bl"][1], 6, True,
           lambda n: "Buckley-Leverett (Section 4.1), N = 200, t = 0.3 (%d steps)" % n)
    for o in (4, 8, 10):
        report("sod%d" % o, spec["sod%d" % o][1], o, False,
               lambda n, o=o: "Order %d, Sod tube N = 200 (%d steps)" % (o, n))
    print("\noracle (%d processes) and GPU wall time %.0f s" % (min(args.jobs, len(jobs)),
                                                             time.time() - t0))


if __name__ == "__main__":
    main()

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
Not collected by pytest (a measurement, about 5 minutes of oracle time); its
output is summarised in profiles/errors_by_config.md.

    python tests/report_errors.py [--n2d 512] [--steps2d 200]
"""
import argparse
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


def grid_of(d):
    sysname = {0: "advection", 1: "euler", 2: "burgers", 3: "buckley_leverett"}[d.system]
    return oracle.make_grid(system=sysname, ndim=d.ndim, nbatch=d.nbatch, nx=d.nx, ny=d.ny,
                            dx=(d.x1 - d.x0) / d.nx,
                            dy=(d.y1 - d.y0) / d.ny if d.ndim == 2 else 1.0,
                            bc_x={0: "transmissive", 1: "periodic"}[d.bc_x],
                            bc_y={0: "transmissive", 1: "periodic"}[d.bc_y], gamma=d.gamma,
                            eps=d.eps, mu0=d.mu0, p=d.p, ai=d.ai, adv_speed=d.adv_speed,
                            order=d.order)


def oracle_spread(w, n_steps, t_final, order=6):
    """The oracle's own rounding floor: the stock run, the run from the input
    times (1 +- 1e-16) and the run in the reversed-summation build (each with
    its own CFL steps)."""
    d = weno.desc_for(w, order=order)
    g = grid_of(d)
    U0 = np.ascontiguousarray(w["U"])

    def go(U):
        t = 0.0
        for _ in range(n_steps):
            if t >= t_final:
                break
            dt = min(float(oracle.cfl_dt(g, U, d.cfl).min()), t_final - t)
            U = oracle.ssprk3_step(g, U, dt)
            t += dt
        return U

    rng = np.random.default_rng(1)
    base = go(U0)
    pert = go(U0 * (1 + 1e-16 * rng.choice([-1.0, 1.0], size=U0.shape)))
    with oracle.rounding_variant("reversed"):
        rev = go(U0)
    return base, pert, rev


def run(w, t_final=None, steps=None, order=6, with_fp32=True):
    """Advance oracle, GPU FP64 (and GPU FP32-recon) with the oracle's steps."""
    d64 = weno.desc_for(w, order=order)
    d32 = weno.desc_for(w, precision="fp32_recon") if with_fp32 else None
    g = grid_of(d64)
    U_o = np.ascontiguousarray(w["U"]).copy()
    A = torch.from_numpy(U_o.copy()).cuda()
    B = torch.from_numpy(U_o.copy()).cuda() if with_fp32 else None
    t, n = 0.0, 0
    while True:
        if steps is not None and n >= steps:
            break
        dt = float(oracle.cfl_dt(g, U_o, d64.cfl).min())
        if t_final is not None:
            if t >= t_final:
                break
            dt = min(dt, t_final - t)
        U_o = oracle.ssprk3_step(g, U_o, dt)
        weno.step(d64, A, dt=dt, sync=False)
        if with_fp32:
            weno.step(d32, B, dt=dt, sync=False)
        t += dt
        n += 1
    torch.cuda.synchronize()
    return U_o, A.cpu().numpy(), (B.cpu().numpy() if with_fp32 else None), t, n


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
    args = ap.parse_args()
    t0 = time.time()
    print("# GPU outputs against the FP64 oracle, every configuration")

    w = wl.advection_sine(n=200)
    U_o, a, b, t, n = run(w, t_final=w["t_final"])
    ex = w["exact"](w["x"], t)
    e_o = np.abs(U_o[0, 0, 0] - ex)
    table("C1 linear advection, N = 200, periodic [-1, 1], t = 2 (%d steps)" % n, U_o, a, b,
          "oracle against the exact solution: L1 (mean) %.2e, Linf %.2e; GPU FP64 against "
          "it: %.2e, %.2e" % (e_o.mean(), e_o.max(), np.abs(a[0, 0, 0] - ex).mean(),
                              np.abs(a[0, 0, 0] - ex).max()),
          spread=oracle_spread(w, n, w["t_final"]))

    w = wl.shock_density(n=1600)
    U_o, a, b, t, n = run(w, t_final=w["t_final"])
    table("C2 1D Euler shock-density, N = 1600 on [-5, 5], t = 1.8 (%d steps)" % n, U_o, a, b,
          spread=oracle_spread(w, n, w["t_final"]))

    w = wl.riemann_batch(nbatch=64, n=1600, seed=2)
    U_o, a, b, t, n = run(w, t_final=w["t_final"])
    m, mx, cnt = riemann_exact_err(w, U_o, t)
    extra = ("oracle density against the exact Riemann solutions (%d problems without "
             "vacuum): mean L1 %.2e, worst problem %.2e" % (cnt, m, mx))
    table("C2 batch of 64 random Riemann problems, N = 1600, t = 0.4 (%d common steps)" % n,
          U_o, a, b, extra, spread=oracle_spread(w, n, w["t_final"]))

    w = wl.quadrant_2d(n=args.n2d, seed=3)
    U_o, a, b, t, n = run(w, steps=args.steps2d)
    table("C3 / C4 2D quadrant (seed 3) at %d^2, %d steps" % (args.n2d, n), U_o, a, b)

    for name, w in (("Burgers (Section 4.1), N = 200, t = 0.2", wl.burgers_sine(n=200)),
                    ("Buckley-Leverett (Section 4.1), N = 200, t = 0.3", wl.buckley_leverett())):
        U_o, a, b, t, n = run(w, t_final=w["t_final"])
        table("%s (%d steps)" % (name, n), U_o, a, b, spread=oracle_spread(w, n, w["t_final"]))

    for order in (4, 8, 10):
        w = wl.shock_tube("sod", n=200)
        U_o, a, _, t, n = run(w, t_final=w["t_final"], order=order, with_fp32=False)
        table("Order %d, Sod tube N = 200 (%d steps)" % (order, n), U_o, a, None,
              spread=oracle_spread(w, n, w["t_final"], order=order))
    print("\noracle and GPU wall time %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()

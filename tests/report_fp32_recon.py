"""Error of the GPU precision modes against the FP64 oracle on a full run.

Runs the seeded quadrant workload (the 2D configuration, seed 3) at n x n for
`steps` SSP-RK3 steps with the oracle's CFL steps, in the oracle (FP64), on
the GPU in FP64 and on the GPU with FP32 reconstruction, and prints the
relative L1 and L_inf error of every conserved component against the oracle.
Not collected by pytest (a measurement, about 4 minutes of oracle time at the
default 512^2 x 200 steps); its printed table is summarised in
profiles/fp32_recon_error_512.md.

    python tests/report_fp32_recon.py [--n 512] [--steps 200]
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

NAMES = ["rho", "rho u", "rho v", "E"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--steps", type=int, default=200)
    args = ap.parse_args()
    w = wl.quadrant_2d(n=args.n, seed=3)
    d64 = weno.desc_for(w)
    d32 = weno.desc_for(w, precision="fp32_recon")
    g = oracle.make_grid(ndim=2, nx=args.n, ny=args.n, dx=(d64.x1 - d64.x0) / args.n,
                         dy=(d64.y1 - d64.y0) / args.n)
    U_o = w["U"].copy()
    A = torch.from_numpy(w["U"]).cuda()
    B = torch.from_numpy(w["U"]).cuda()
    t0 = time.time()
    for _ in range(args.steps):
        dt = float(oracle.cfl_dt(g, U_o, d64.cfl)[0])
        U_o = oracle.ssprk3_step(g, U_o, dt)
        weno.step(d64, A, dt=dt, sync=False)
        weno.step(d32, B, dt=dt, sync=False)
    torch.cuda.synchronize()
    el = time.time() - t0
    a, b = A.cpu().numpy(), B.cpu().numpy()
    print("quadrant %dx%d, %d steps (oracle CFL steps), oracle wall %.0f s" % (args.n, args.n, args.steps, el))
    print("| component | FP64 GPU rel L1 | FP64 GPU rel Linf | FP32-recon rel L1 | FP32-recon rel Linf |")
    print("|---|---|---|---|---|")
    for k in range(4):
        ref = U_o[0, k]
        l1 = lambda x: np.abs(x[0, k] - ref).sum() / np.abs(ref).sum()
        li = lambda x: np.abs(x[0, k] - ref).max() / np.abs(ref).max()
        print("| %s | %.2e | %.2e | %.2e | %.2e |" % (NAMES[k], l1(a), li(a), l1(b), li(b)))


if __name__ == "__main__":
    main()

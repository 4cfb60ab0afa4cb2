"""Seeded random parity sweep: many small problems of random shape, batch,
boundary, system, scheme order, weight options and precision, each checked
against the oracle -- the right-hand side and one SSP-RK3 step at 1e-12
relative L_inf for FP64; for FP32 reconstruction the right-hand side within
1e-5 relative L_inf and the step within 1e-6 relative L1.  The
shapes include ragged tiles, grids smaller than the stencil and batches."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_26272_gb300 import weno
from paper_2603_26272_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

N_CASES = 60


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_err(a, b):
    scale_all = max(np.abs(b).max(), 1e-300)
    worst = 0.0
    for k in range(a.shape[1]):
        s = np.abs(b[:, k]).max()
        if s <= 1e-14 * scale_all:
            s = scale_all
        worst = max(worst, np.abs(a[:, k] - b[:, k]).max() / s)
    return worst


def rel_l1(a, b):
    return np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-300)


def make_case(k):
    rng = np.random.default_rng(1000 + k)
    system = rng.choice(["euler1d", "euler2d", "euler2d", "advection", "burgers", "bl"])
    bc = str(rng.choice(["transmissive", "periodic"]))
    order = int(rng.choice([6, 6, 6, 4, 8, 10]))
    ai = bool(rng.random() < 0.8)
    p = float(rng.choice([1.0, 1.0, 1.5, 2.0]))
    single = bool(rng.random() < 0.2)
    prec = "fp32_recon" if (ai and order == 6 and rng.random() < 0.3) else "fp64"
    if system == "euler2d":
        nx, ny = int(rng.integers(1, 70)), int(rng.integers(1, 70))
        nb = int(rng.integers(1, 4))
        Us = []
        for b in range(nb):
            q = wl.quadrant_2d(n=max(nx, ny), seed=int(rng.integers(1 << 30)))
            Us.append(q["U"][:, :, :ny, :nx])
        w = {"system": "euler", "ndim": 2, "U": np.ascontiguousarray(np.concatenate(Us, 0)),
             "bc": bc, "domain": (0.0, 1.0)}
        d = weno.make_desc(system="euler", ndim=2, nbatch=nb, nx=nx, ny=ny, x1=nx / 64.0,
                           y1=ny / 64.0, bc_x=bc, bc_y=bc, ai=ai, p=p, precision=prec,
                           alpha_mode="single" if single else "field", order=order)
    elif system == "euler1d":
        n = int(rng.integers(1, 400))
        nb = int(rng.integers(1, 6))
        w = wl.riemann_batch(nbatch=nb, n=n, seed=int(rng.integers(1 << 30)))
        d = weno.make_desc(system="euler", ndim=1, nbatch=nb, nx=n, x0=-5.0, x1=5.0, bc_x=bc,
                           ai=ai, p=p, precision=prec, alpha_mode="single" if single else "field",
                           order=order)
    else:
        n = int(rng.integers(1, 400))
        x = (np.arange(n) + 0.5) / n
        if system == "bl":  # saturations in [0, 1] with a jump
            u = np.clip(0.5 + 0.5 * np.sin(2 * np.pi * (x + rng.random()))
                        + 0.3 * (x > rng.random()), 0.0, 1.0)
            sysname = "buckley_leverett"
        else:
            u = np.sin(2 * np.pi * x + rng.random()) + (x > rng.random()) * rng.uniform(-1, 1)
            sysname = "advection" if system == "advection" else "burgers"
        w = {"U": u.reshape(1, 1, 1, n)}
        d = weno.make_desc(system=sysname, ndim=1, nx=n, bc_x=bc, ai=ai, p=p, precision=prec,
                           adv_speed=float(rng.choice([1.0, -0.7])), order=order)
    return d, np.ascontiguousarray(w["U"], dtype=np.float64)


def grid_of(d):
    sysname = {0: "advection", 1: "euler", 2: "burgers", 3: "buckley_leverett"}[d.system]
    return oracle.make_grid(system=sysname, ndim=d.ndim, nbatch=d.nbatch, nx=d.nx, ny=d.ny,
                            dx=(d.x1 - d.x0) / d.nx,
                            dy=(d.y1 - d.y0) / d.ny if d.ndim == 2 else 1.0,
                            bc_x={0: "transmissive", 1: "periodic"}[d.bc_x],
                            bc_y={0: "transmissive", 1: "periodic"}[d.bc_y], gamma=d.gamma,
                            eps=d.eps, mu0=d.mu0, p=d.p, ai=d.ai,
                            alpha_mode={0: "field", 1: "single"}[d.alpha_mode],
                            adv_speed=d.adv_speed, order=d.order or 6)


@pytest.mark.parametrize("k", range(N_CASES))
def test_random_case_matches_oracle(k):
    d, U = make_case(k)
    g = grid_of(d)
    L_o = oracle.rhs(g, U)
    dt = oracle.cfl_dt(g, U, d.cfl)
    U1_o = oracle.ssprk3_step(g, U, dt)
    Ug = torch.from_numpy(U.copy()).cuda()
    L_g = weno.rhs(d, Ug).cpu().numpy()
    used = weno.step(d, Ug)
    U1_g = Ug.cpu().numpy()
    np.testing.assert_allclose(used, dt, rtol=1e-12, atol=0)
    if d.precision == weno.PRECISIONS["fp64"]:
        assert rel_err(L_g, L_o) <= 1e-12, (k, rel_err(L_g, L_o))
        assert rel_err(U1_g, U1_o) <= 1e-12, (k, rel_err(U1_g, U1_o))
    else:  # the bounds of the FP32-reconstruction tests: per stage, per step
        assert rel_err(L_g, L_o) <= 1e-5, (k, rel_err(L_g, L_o))
        assert rel_l1(U1_g, U1_o) <= 1e-6, (k, rel_l1(U1_g, U1_o))

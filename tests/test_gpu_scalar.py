"""GPU parity on the scalar equations of Section 4.1 (Table 5): Burgers and
Buckley-Leverett (and linear advection), FP64 path against the oracle per
stage (1e-12) and over full runs (1e-10, or 4x the oracle's own spread under
rounding-level input noise or reversed summation order), and the
FP32-reconstruction mode's relative L1 error (<= 1e-6)."""
import numpy as np
import pytest
import torch

import oracle
import rounding_spread
from paper_2603_26272_gb300 import weno
from paper_2603_26272_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_linf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _grid(w, d):
    return oracle.make_grid(system=w["system"], ndim=1, nx=d.nx, dx=(d.x1 - d.x0) / d.nx,
                            bc_x=w["bc"])


CASES = [("burgers", wl.burgers_sine()), ("burgers_400", wl.burgers_sine(n=400)),
         ("bl_paper", wl.buckley_leverett()), ("bl_riemann", wl.buckley_riemann(n=300)),
         ("advection", wl.advection_sine(n=130))]


@pytest.mark.parametrize("name,w", CASES, ids=[c[0] for c in CASES])
def test_scalar_rhs_speeds_and_step(name, w):
    d = weno.desc_for(w)
    g = _grid(w, d)
    U = np.ascontiguousarray(w["U"])
    L_o = oracle.rhs(g, U)
    Ug = torch.from_numpy(U).cuda()
    L_g = weno.rhs(d, Ug).cpu().numpy()
    assert rel_linf(L_g, L_o) <= 1e-12, name
    al, dt = weno.wavespeeds(d, Ug)
    assert al.cpu().numpy()[0, 0, 0] == pytest.approx(oracle.alpha(g, U)[0, 0, 0], rel=1e-12)
    assert dt.cpu().numpy()[0] == pytest.approx(oracle.cfl_dt(g, U, d.cfl)[0], rel=1e-12)
    dt_o = oracle.cfl_dt(g, U, d.cfl)
    U_o = oracle.ssprk3_step(g, U, dt_o)
    weno.step(d, Ug)
    assert rel_linf(Ug.cpu().numpy(), U_o) <= 1e-12, name


@pytest.mark.parametrize("name,w", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_scalar_full_runs(name, w):
    d = weno.desc_for(w)
    g = _grid(w, d)
    U_o, t_o, n_o = oracle.solve(g, w["U"], d.cfl, w["t_final"])
    tol = rounding_spread.run_bound(lambda V: oracle.solve(g, V, d.cfl, w["t_final"])[0],
                                    w["U"], rel_linf)
    Ug = torch.from_numpy(w["U"]).cuda()
    t_g, n_g = weno.solve(d, Ug, w["t_final"])
    assert n_g[0] == n_o[0] and t_g[0] == t_o[0]
    assert rel_linf(Ug.cpu().numpy(), U_o) <= tol, name
    d32 = weno.desc_for(w, precision="fp32_recon")
    U32 = torch.from_numpy(w["U"]).cuda()
    weno.solve(d32, U32, w["t_final"])
    l1 = np.abs(U32.cpu().numpy() - U_o).sum() / np.abs(U_o).sum()
    assert l1 <= 1e-6, (name, l1)

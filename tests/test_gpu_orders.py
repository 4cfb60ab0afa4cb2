"""GPU parity of the central-upwind schemes of order 4, 8 and 10 (r = 2, 4, 5;
the tables of the Appendix with the weights of eqs. (16)-(22)) against the
oracle: the right-hand side and one SSP-RK3 step at 1e-12 relative L_inf,
full runs at 1e-10 (or 4x the oracle's own spread under rounding-level input
noise or reversed summation order), on 1D Euler, the scalar equations and 2D Euler, with ragged tiles,
grids smaller than the stencil and both boundary kinds."""
import numpy as np
import pytest
import torch

import oracle
import rounding_spread
from paper_2603_26272_gb300 import weno
from paper_2603_26272_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STAGE_TOL = 1e-12
RUN_TOL = 1e-10
ORDERS = (4, 8, 10)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    weno.lib()
    oracle.lib()


def rel_err(a, b):
    """max over components of max|a - b| / max|b| (a near-zero component is
    measured against the largest one)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale_all = max(np.abs(b).max(), 1e-300)
    worst = 0.0
    for k in range(a.shape[1]):
        s = np.abs(b[:, k]).max()
        if s <= 1e-14 * scale_all:
            s = scale_all
        worst = max(worst, np.abs(a[:, k] - b[:, k]).max() / s)
    return worst


def grid_of(w, d):
    sysname = {0: "advection", 1: "euler", 2: "burgers", 3: "buckley_leverett"}[d.system]
    return oracle.make_grid(system=sysname, ndim=d.ndim, nbatch=d.nbatch, nx=d.nx, ny=d.ny,
                            dx=(d.x1 - d.x0) / d.nx,
                            dy=(d.y1 - d.y0) / d.ny if d.ndim == 2 else 1.0,
                            bc_x={0: "transmissive", 1: "periodic"}[d.bc_x],
                            bc_y={0: "transmissive", 1: "periodic"}[d.bc_y], gamma=d.gamma,
                            eps=d.eps, mu0=d.mu0, p=d.p, ai=d.ai,
                            alpha_mode={0: "field", 1: "single"}[d.alpha_mode],
                            adv_speed=d.adv_speed, order=d.order)


def desc_of(w, order, **kw):
    d = weno.desc_for(w, order=order, **kw)
    if w["ndim"] == 2 and "dx" in w:  # sub-sliced grids keep the cell size
        d.x0, d.x1 = 0.0, d.nx * w["dx"]
        d.y0, d.y1 = 0.0, d.ny * w["dy"]
    return d


def cut2d(w, nx, ny):
    w = dict(w)
    w["U"] = np.ascontiguousarray(w["U"][:, :, :ny, :nx])
    return w


def cases():
    out = [("shock_density300", wl.shock_density(n=300), {}),
           ("riemann_batch", wl.riemann_batch(nbatch=5, n=260, seed=2), {}),
           ("sod_n3", wl.shock_tube("sod", n=3), {}),
           ("sod_n128", wl.shock_tube("sod", n=128), {}),
           ("periodic_n4", wl.smooth_euler_1d(n=4, seed=3), {}),
           ("periodic_n64", wl.smooth_euler_1d(n=64, seed=1), {}),
           ("advection131", wl.advection_sine(n=131), {}),
           ("advection_noai_p2", wl.advection_sine(n=90), {"ai": False, "p": 2.0}),
           ("burgers", wl.burgers_sine(n=200), {}),
           ("buckley_leverett", wl.buckley_leverett(n=200), {}),
           ("quadrant70", wl.quadrant_2d(n=70, seed=3), {}),
           ("quadrant40x27", cut2d(wl.quadrant_2d(n=40, seed=4), 40, 27), {}),
           ("smooth_periodic", wl.random_smooth_2d(nx=36, ny=30, seed=2), {}),
           ("tiny5x3", cut2d(wl.quadrant_2d(n=5, seed=7), 5, 3), {}),
           ("config3_noai", wl.config3_2d(n=40), {"ai": False}),
           ("quadrant_p15_single", wl.quadrant_2d(n=34, seed=6),
            {"p": 1.5, "alpha_mode": "single"})]
    return [(o, n, w, kw) for o in ORDERS for (n, w, kw) in out]


CASES = cases()
IDS = ["o%d-%s" % (c[0], c[1]) for c in CASES]


@pytest.mark.parametrize("order,name,w,kw", CASES, ids=IDS)
def test_rhs_and_step_match_oracle(order, name, w, kw):
    d = desc_of(w, order, **kw)
    g = grid_of(w, d)
    U = np.ascontiguousarray(w["U"])
    L_o = oracle.rhs(g, U)
    Ug = torch.from_numpy(U).cuda()
    L_g = weno.rhs(d, Ug).cpu().numpy()
    assert rel_err(L_g, L_o) <= STAGE_TOL, (order, name)
    dt = oracle.cfl_dt(g, U, d.cfl)
    U_o = oracle.ssprk3_step(g, U, dt)
    used = weno.step(d, Ug)
    np.testing.assert_allclose(used, dt, rtol=STAGE_TOL, atol=0)
    assert rel_err(Ug.cpu().numpy(), U_o) <= STAGE_TOL, (order, name)


def test_orders_differ():
    """The order field reaches the kernels: on a smooth problem the four
    schemes give four different right-hand sides."""
    w = wl.random_smooth_2d(nx=32, ny=32, seed=5)
    Ug = torch.from_numpy(np.ascontiguousarray(w["U"])).cuda()
    outs = [weno.rhs(desc_of(w, o), Ug).cpu().numpy() for o in (4, 6, 8, 10)]
    for i in range(4):
        for j in range(i + 1, 4):
            assert np.abs(outs[i] - outs[j]).max() > 1e-10


RUNS = [("sod", wl.shock_tube("sod", n=200)), ("lax", wl.shock_tube("lax", n=200)),
        ("burgers", wl.burgers_sine(n=200)), ("buckley_leverett", wl.buckley_leverett(n=150))]


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("name,w", RUNS, ids=[r[0] for r in RUNS])
def test_full_runs_1d(order, name, w):
    d = desc_of(w, order)
    g = grid_of(w, d)
    U_o, t_o, n_o = oracle.solve(g, w["U"], d.cfl, w["t_final"])
    tol = rounding_spread.run_bound(lambda V: oracle.solve(g, V, d.cfl, w["t_final"])[0],
                                    w["U"], rel_err, RUN_TOL)
    Ug = torch.from_numpy(np.ascontiguousarray(w["U"])).cuda()
    t_g, n_g = weno.solve(d, Ug, w["t_final"])
    assert list(n_g) == list(n_o)
    np.testing.assert_array_equal(np.asarray(t_g), t_o)
    assert rel_err(Ug.cpu().numpy(), U_o) <= tol, (order, name)


@pytest.mark.parametrize("order", ORDERS)
def test_full_run_2d(order):
    w = wl.quadrant_2d(n=40, seed=3)
    d = desc_of(w, order)
    g = grid_of(w, d)
    U0 = np.ascontiguousarray(w["U"])

    def oracle_run(U):
        for _ in range(30):
            U = oracle.ssprk3_step(g, U, oracle.cfl_dt(g, U, d.cfl))
        return U

    # the tenth-order run amplifies rounding-level input noise to ~2e-10 in
    # the oracle itself; the bound is 4x the oracle's own spread where that
    # exceeds 1e-10
    tol = rounding_spread.run_bound(oracle_run, U0, rel_err, RUN_TOL)
    U_o = U0
    Ug = torch.from_numpy(U0).cuda()
    for k in range(30):
        dt = oracle.cfl_dt(g, U_o, d.cfl)
        U_o = oracle.ssprk3_step(g, U_o, dt)
        used = weno.step(d, Ug)
        # after the first step dt comes from states that already differ by
        # the accumulated rounding of the run, so it is held to the run bound
        np.testing.assert_allclose(used, dt, rtol=STAGE_TOL if k == 0 else tol)
    assert rel_err(Ug.cpu().numpy(), U_o) <= tol


@pytest.mark.parametrize("order", ORDERS)
def test_sampled_cells_of_a_large_grid(order):
    """A 1024^2 quadrant grid (many full tiles, the launch shape of large
    problems): L(U) on sampled cells against the oracle cell by cell."""
    w = wl.quadrant_2d(n=1024, seed=3)
    d = desc_of(w, order)
    g = grid_of(w, d)
    U = w["U"]
    Ug = torch.from_numpy(U).cuda()
    L_g = weno.rhs(d, Ug).cpu().numpy()
    al = oracle.alpha(g, U)
    n = 1024
    rng = np.random.default_rng(order)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n // 2, n // 2 - 1)]
    pts += [(int(j), int(i)) for j, i in rng.integers(0, n, size=(30, 2))]
    pts += [(int(j), n // 2 + int(o)) for j, o in zip(rng.integers(0, n, 20), rng.integers(-6, 6, 20))]
    scale = np.abs(L_g[0]).reshape(4, -1).max(axis=1)
    scale = np.where(scale <= 1e-14 * scale.max(), scale.max(), scale)
    for (j, i) in pts:
        lo = oracle.rhs_cell(g, U, al, 0, j, i)
        assert (np.abs(L_g[0, :, j, i] - lo) / scale).max() <= STAGE_TOL, (order, j, i)


def test_engine_and_fp32_recon_refuse_other_orders():
    w = wl.shock_tube("sod", n=64)
    d = desc_of(w, 8, precision="fp32_recon")
    with pytest.raises(weno.WenoError):
        weno.workspace_bytes(d)
    from paper_2603_26272_gb300 import serve
    eng = serve.Engine(64 << 20, max_slots=4, max_tiles=1024)
    try:
        with pytest.raises(weno.WenoError):
            eng.admit(desc_of(w, 8), w["U"], 0.1)
        assert eng.admit(desc_of(w, 6), w["U"], 0.1) is not None
    finally:
        eng.close()

"""Pin the oracle's right-hand side and SSP-RK3 stepping (Sections 2 and 4).

What is fixed independently of any implementation:
* eq. (5) is a telescoping flux difference: with periodic boundaries the cell
  sum of L(U) is zero; with constant far-field states it equals the boundary
  flux budget -(F(U_R) - F(U_L)).
* A uniform state has L(U) = 0.
* Reflection x -> -x, u -> -u maps the scheme onto itself (the negative flux is
  the mirror image of the positive one, Section 2 after eq. (6)).
* 2D data independent of y reduce to the 1D scheme row by row; swapping x and
  y (with u and v) transposes the right-hand side.
* Smooth advection converges at sixth order in space (Section 3.1, Table 2:
  p = 1 suffices for critical points of order <= 2) and third order in time
  (the TVD Runge-Kutta of the Section 4 preamble).
* Riemann problems converge to the exact solution (Section 4.2).
"""
import numpy as np
import pytest

import oracle
from paper_2603_26272_gb300 import workloads as wl


def _grid1(w, **kw):
    return oracle.make_grid(system=w["system"], ndim=1, nbatch=w["U"].shape[0], nx=w["n"],
                            dx=w["dx"], bc_x=w["bc"], **kw)


def test_uniform_state_is_steady():
    U = wl.cons_2d(np.full((8, 9), 0.7), np.full((8, 9), 0.3), np.full((8, 9), -0.2),
                   np.full((8, 9), 1.1)).reshape(1, 4, 8, 9)
    for bc in ("periodic", "transmissive"):
        g = oracle.make_grid(ndim=2, nx=9, ny=8, dx=0.1, dy=0.2, bc_x=bc, bc_y=bc)
        L = oracle.rhs(g, U)
        assert np.abs(L).max() < 1e-13


@pytest.mark.parametrize("ai", [0, 1])
def test_periodic_conservation_1d(ai):
    w = wl.smooth_euler_1d(n=64, seed=1)
    U = w["U"].copy()
    U[0, :, 0, 20:40] *= 1.3  # add two jumps
    g = _grid1(w, ai=ai)
    L = oracle.rhs(g, U)
    for k in range(3):
        assert abs(L[0, k].sum()) <= 1e-13 * np.abs(L[0, k]).sum()


def test_periodic_conservation_2d():
    w = wl.random_smooth_2d(nx=24, ny=20, seed=2)
    U = w["U"].copy()
    U[0, :, 5:12, 3:15] *= 1.2
    g = oracle.make_grid(ndim=2, nx=24, ny=20, dx=w["dx"], dy=w["dy"], bc_x="periodic",
                         bc_y="periodic")
    L = oracle.rhs(g, U)
    for k in range(4):
        assert abs(L[0, k].sum()) <= 1e-13 * np.abs(L[0, k]).sum()


def test_transmissive_flux_budget():
    w = wl.riemann_1d((1.0, 0.75, 1.0), (0.125, 0.0, 0.1), x0=0.0, n=120)
    g = _grid1(w)
    L = oracle.rhs(g, w["U"])
    def flux(r, u, p):
        E = p / 0.4 + 0.5 * r * u * u
        return np.array([r * u, r * u * u + p, (E + p) * u])
    budget = -(flux(0.125, 0.0, 0.1) - flux(1.0, 0.75, 1.0))
    got = L[0, :, 0, :].sum(axis=1) * w["dx"]
    np.testing.assert_allclose(got, budget, rtol=0, atol=1e-12)


def test_mirror_symmetry_1d():
    w = wl.shock_density(n=96)
    U = w["U"]
    g = _grid1(w)
    L = oracle.rhs(g, U)
    Um = U[:, :, :, ::-1].copy()
    Um[:, 1] *= -1.0
    Lm = oracle.rhs(g, Um)
    Lb = Lm[:, :, :, ::-1].copy()
    Lb[:, 1] *= -1.0
    scale = np.abs(L).max()
    assert np.abs(Lb - L).max() <= 1e-13 * scale


def test_2d_reduces_to_1d_and_transposes():
    w1 = wl.shock_density(n=80)
    g1 = _grid1(w1)
    L1 = oracle.rhs(g1, w1["U"])
    ny = 7
    U1 = w1["U"][0, :, 0, :]
    U2 = np.zeros((1, 4, ny, 80))
    U2[0, 0] = U1[0]
    U2[0, 1] = U1[1]
    U2[0, 3] = U1[2]
    for bcy in ("transmissive", "periodic"):
        g2 = oracle.make_grid(ndim=2, nx=80, ny=ny, dx=w1["dx"], dy=0.37, bc_y=bcy)
        L2 = oracle.rhs(g2, U2)
        scale = np.abs(L1).max()
        for j in range(ny):
            assert np.abs(L2[0, [0, 1, 3], j, :] - L1[0, :, 0, :]).max() <= 1e-13 * scale
        assert np.abs(L2[0, 2]).max() <= 1e-13 * scale
    # transpose: swap axes and the momentum components
    w = wl.quadrant_2d(n=24, seed=5)
    U = w["U"]
    g = oracle.make_grid(ndim=2, nx=24, ny=24, dx=w["dx"], dy=w["dx"])
    L = oracle.rhs(g, U)
    UT = U[:, [0, 2, 1, 3]].transpose(0, 1, 3, 2).copy()
    LT = oracle.rhs(g, UT)[:, [0, 2, 1, 3]].transpose(0, 1, 3, 2)
    assert np.abs(LT - L).max() <= 1e-13 * np.abs(L).max()


def _advect_error(n, dt_rule, t_final=2.0, cfl=0.5):
    w = wl.advection_sine(n=n, cfl=cfl, t_final=t_final)
    g = _grid1(w)
    dx = w["dx"]
    dt = cfl * dx * dx if dt_rule == "dx2" else cfl * dx
    steps = int(np.ceil(t_final / dt - 1e-12))
    dt = t_final / steps
    U = w["U"].copy()
    for _ in range(steps):
        U = oracle.ssprk3_step(g, U, dt)
    return np.abs(U[0, 0, 0] - w["exact"](w["x"], t_final)).max(), U, w


@pytest.mark.slow
def test_advection_sixth_order_in_space():
    errs = [_advect_error(n, "dx2")[0] for n in (20, 40, 80)]
    orders = [np.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert orders[-1] > 5.5, (errs, orders)


def test_advection_config_and_conservation():
    e, U, w = _advect_error(200, "dx")
    assert e < 1e-5  # dominated by the O(dt^3) time error at dt = 0.5 dx
    assert abs(U.sum() - w["U"].sum()) <= 1e-13 * np.abs(w["U"]).sum()


def test_ssprk3_is_third_order_in_time():
    # Same spatial operator, several dt: the time error falls like dt^3.
    w = wl.advection_sine(n=40)
    g = _grid1(w)
    T = 0.5
    def run(steps):
        U = w["U"].copy()
        for _ in range(steps):
            U = oracle.ssprk3_step(g, U, T / steps)
        return U
    ref = run(2000)
    errs = [np.abs(run(s) - ref).max() for s in (25, 50, 100)]
    orders = [np.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert min(orders) > 2.8, orders


def test_cfl_dt_rule():
    rho, u, v, p = 0.8, 0.3, -0.6, 1.2
    U = wl.cons_2d(np.full((4, 5), rho), np.full((4, 5), u), np.full((4, 5), v),
                   np.full((4, 5), p)).reshape(1, 4, 4, 5)
    g = oracle.make_grid(ndim=2, nx=5, ny=4, dx=0.2, dy=0.25)
    c = np.sqrt(1.4 * p / rho)
    want = 0.5 / ((abs(u) + c) / 0.2 + (abs(v) + c) / 0.25)
    assert oracle.cfl_dt(g, U, 0.5)[0] == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("name", ["sod", "lax", "123"])
def test_shock_tubes_converge_to_exact(name):
    errs = []
    for n in (200, 400):
        w = wl.shock_tube(name, n=n)
        g = _grid1(w)
        U, t, _ = oracle.solve(g, w["U"], w["cfl"], w["t_final"])
        assert t[0] == w["t_final"]
        rho, u, p, star = oracle.riemann_exact(w["left"], w["right"], w["x"], w["t_final"])
        errs.append(np.abs(U[0, 0, 0] - rho).mean())
        if name != "123":
            # the shock sits where the numerical density crosses the mean of the
            # exact pre- and post-shock densities, within 2 dx
            jump = np.abs(np.diff(rho))
            k = int(np.argmax(jump))
            mid = 0.5 * (rho[k] + rho[k + 1])
            num = U[0, 0, 0]
            lo, hi = max(k - 20, 0), min(k + 21, n - 1)
            s = np.where(np.diff(np.sign(num[lo:hi] - mid)) != 0)[0]
            assert s.size > 0
            xs_num = w["x"][lo + s[0]]
            assert abs(xs_num - 0.5 * (w["x"][k] + w["x"][k + 1])) <= 2 * w["dx"]
    assert errs[1] < errs[0]
    assert errs[0] < {"sod": 0.01, "lax": 0.03, "123": 0.02}[name]


@pytest.mark.parametrize("seed", [3, 4])
def test_quadrant_problem_stays_physical(seed):
    w = wl.quadrant_2d(n=32, seed=seed)
    g = oracle.make_grid(ndim=2, nx=32, ny=32, dx=w["dx"], dy=w["dx"])
    U, t, steps = oracle.solve(g, w["U"], w["cfl"], 1.0, max_steps=100, allow_max_steps=True)
    assert steps[0] == 100
    assert np.isfinite(U).all() and U[0, 0].min() > 0

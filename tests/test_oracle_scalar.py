"""Pin the oracle on the scalar equations of Section 4.1 (Table 5).

* Burgers, u0 = 1/2 + sin(2 pi x): before the shock forms (t < 1/(2 pi)) the
  exact solution follows the characteristics, u = u0(x - u t); the scheme must
  converge to it at high order.  After it (T = 0.2) the mass is conserved and,
  since u - 1/2 is odd about x = 1/2 in the frame moving at speed 1/2, the
  shock sits at x = 1/2 + t/2.
* Buckley-Leverett, f = u^2 / (u^2 + (1 - u)^2 / 4): the Riemann problem
  1 | 0 has the textbook entropy solution built from the upper concave
  envelope of f -- a fan through the concave part from u = 1 down to the
  tangent point u* (u* f'(u*) = f(u*)) and a shock from u* to 0 at speed
  f'(u*).  The paper's two-jump problem keeps 0 <= u <= 1 and its mass.
"""
import numpy as np
import pytest

import oracle
from paper_2603_26272_gb300 import workloads as wl


def _grid(w):
    return oracle.make_grid(system=w["system"], ndim=1, nx=w["n"], dx=w["dx"], bc_x=w["bc"])


def _burgers_exact(x, t):
    u = 0.5 + np.sin(2 * np.pi * x)
    for _ in range(60):  # Newton on u - u0(x - u t) = 0
        xi = x - u * t
        F = u - (0.5 + np.sin(2 * np.pi * xi))
        dF = 1.0 + 2 * np.pi * np.cos(2 * np.pi * xi) * t
        u = u - F / dF
    return u


def test_burgers_smooth_convergence():
    errs = []
    for n in (40, 80, 160):
        w = wl.burgers_sine(n=n)
        g = _grid(w)
        T = 0.1
        dt0 = 0.2 * w["dx"] ** 2
        steps = int(np.ceil(T / dt0))
        U = w["U"].copy()
        for _ in range(steps):
            U = oracle.ssprk3_step(g, U, T / steps)
        errs.append(np.abs(U[0, 0, 0] - _burgers_exact(w["x"], T)).max())
    orders = [np.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert orders[-1] > 4.5, (errs, orders)


def test_burgers_shock_conservation_and_position():
    w = wl.burgers_sine(n=200)
    U, t, n = oracle.solve(_grid(w), w["U"], w["cfl"], w["t_final"])
    u = U[0, 0, 0]
    assert abs(u.sum() - w["U"].sum()) <= 1e-13 * np.abs(w["U"]).sum()
    assert u.min() > -0.5 - 1e-3 and u.max() < 1.5 + 1e-3
    k = int(np.argmin(np.diff(u)))  # steepest descent: the shock
    xs = 0.5 * (w["x"][k] + w["x"][k + 1])
    assert abs(xs - (0.5 + 0.5 * w["t_final"])) <= 2 * w["dx"]


def _bl_f(u):
    return u * u / (u * u + 0.25 * (1 - u) ** 2)


def _bl_df(u):
    D = u * u + 0.25 * (1 - u) ** 2
    return 0.5 * u * (1 - u) / D ** 2


def _bisect(fun, lo, hi, n=200):
    flo = fun(lo)
    for _ in range(n):
        mid = 0.5 * (lo + hi)
        if (fun(mid) > 0) == (flo > 0):
            lo, flo = mid, fun(mid)
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _bl_riemann_exact(x, t):
    # tangent point of the line from the origin: u f'(u) - f(u) = 0 on (0.2, 1)
    us = _bisect(lambda u: u * _bl_df(u) - _bl_f(u), 0.2, 1.0)
    s = _bl_df(us)
    out = np.zeros_like(x)
    for k, xi in enumerate(x / t):
        if xi < 0:
            out[k] = 1.0
        elif xi <= s:  # fan: f'(u) = xi on [us, 1], f' decreasing there
            out[k] = _bisect(lambda u: _bl_df(u) - xi, us, 1.0)
        else:
            out[k] = 0.0
    return out, us, s


def test_buckley_leverett_riemann_converges_to_exact():
    errs = []
    for n in (200, 400, 800):
        w = wl.buckley_riemann(n=n)
        U, _, _ = oracle.solve(_grid(w), w["U"], w["cfl"], w["t_final"])
        ex, us, s = _bl_riemann_exact(w["x"], w["t_final"])
        errs.append(np.abs(U[0, 0, 0] - ex).mean())
    # closed forms of the tangent construction for f = u^2/(u^2 + a(1-u)^2),
    # a = 1/4: u* = sqrt(a/(1+a)) = 1/sqrt(5), shock speed (1 + sqrt(5))/2
    assert us == pytest.approx(1 / np.sqrt(5), abs=1e-12)
    assert s == pytest.approx((1 + np.sqrt(5)) / 2, abs=1e-9)
    assert errs[0] < 0.005 and errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1], errs


def test_buckley_leverett_paper_problem_bounds_and_mass():
    w = wl.buckley_leverett()
    g = _grid(w)
    U, t, n = oracle.solve(g, w["U"], w["cfl"], w["t_final"])
    u = U[0, 0, 0]
    assert u.min() > -1e-6 and u.max() < 1 + 1e-6
    assert abs(u.sum() - w["U"].sum()) <= 1e-12 * w["U"].sum()
    # eq. (6) for the nonconvex flux: the speed peaks inside (0, 1)
    al = oracle.alpha(g, w["U"])[0, 0, 0]
    uu = np.linspace(0, 1, 200001)
    assert al == pytest.approx(_bl_df(uu).max(), rel=1e-9)

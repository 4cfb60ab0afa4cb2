"""Pin the oracle's fourth-, eighth- and tenth-order schemes (Appendix).

* Every printed table (c_2r, c_k with the rev() relations, d, the smoothness
  matrices B_k and B_d, c_tau) is re-derived in exact arithmetic from the
  definitions of Section 2 (eqs. (8)-(9), (12), (15), (17)), as for r = 3.
  (The fourth-order downwind substencil is S_2; the Appendix text names it
  S_3 once -- a misprint, its own beta formula uses S_2.)
* The generic routine with the r = 3 tables is bit for bit the pinned
  WENO-ZA6 routine.
* Data that are a polynomial of degree <= 2r - 2 have tau = 0, so the flux is
  the central flux <c_2r, f>.
* On smooth data without critical points the operator converges at order 2r.
* The Euler and scalar right-hand sides of every order conserve mass.
"""
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2603_26272_gb300 import workloads as wl

X = sp.Symbol("x")


def _interp(nodes):
    m = len(nodes)
    a = sp.symbols("a0:%d" % m)
    f = sp.symbols("f0:%d" % m)
    p = sum(a[n] * X ** n for n in range(m))
    sol = sp.solve([sp.integrate(p, (X, l - sp.Rational(1, 2), l + sp.Rational(1, 2))) - f[k]
                    for k, l in enumerate(nodes)], a, dict=True)[0]
    return sp.expand(p.subs(sol)), f


def _frac(x, den):
    return Fraction(x).limit_denominator(den)


def _q(c):
    c = sp.Rational(sp.simplify(c))
    return Fraction(int(c.p), int(c.q))


@pytest.mark.parametrize("order", [4, 8, 10])
def test_appendix_tables_from_definitions(order):
    r = order // 2
    t = oracle.coefficients_r(order)
    big = 10 ** 7
    # central flux and candidates: cell-average interpolation evaluated at 1/2
    p, f = _interp(list(range(-r + 1, r + 1)))
    c2r = [sp.expand(p.subs(X, sp.Rational(1, 2))).coeff(v) for v in f]
    assert [_frac(v, big) for v in t["c2r"]] == [_q(c) for c in c2r]
    for k in range(r + 1):
        p, f = _interp(list(range(-r + 1 + k, k + 1)))
        ck = [sp.expand(p.subs(X, sp.Rational(1, 2))).coeff(v) for v in f]
        assert [_frac(v, big) for v in t["ck"][k]] == [_q(c) for c in ck]
    # ideal weights C(r,k)^2 / C(2r,r), and sum d_k c_k = c_2r exactly
    assert [_frac(v, big) for v in t["d"]] == [Fraction(sp.binomial(r, k) ** 2, sp.binomial(2 * r, r))
                                              for k in range(r + 1)]
    dd = [_frac(v, big) for v in t["d"]]
    ck = [[_frac(v, big) for v in row] for row in t["ck"]]
    comb = [sum(dd[k] * ck[k][j - k] for k in range(r + 1) if k <= j <= k + r - 1) for j in range(2 * r)]
    assert comb == [_frac(v, big) for v in t["c2r"]]
    # smoothness matrices from eq. (15): B_0..B_{r-1} on S_k, B_d on S_r over I_i
    for k in range(r + 1):
        nodes = list(range(-r + 1 + k, k + 1))
        p, f = _interp(nodes)
        beta = sum(sp.integrate(sp.diff(p, X, l) ** 2, (X, -sp.Rational(1, 2), sp.Rational(1, 2)))
                   for l in range(1, r))
        beta = sp.expand(beta)
        for a in range(r):
            for b in range(r):
                want = beta.coeff(f[a], 2) if a == b else beta.coeff(f[a], 1).coeff(f[b], 1) / 2
                assert _frac(t["B"][k][a][b], big) == _q(want), (k, a, b)
    # c_tau: annihilates degree <= 2r-2, gives (2r-1)! on j^(2r-1)
    j = np.arange(2 * r, dtype=np.float64)
    for deg in range(2 * r - 1):
        assert np.dot(t["ctau"], j ** deg) == 0.0
    assert np.dot(t["ctau"], j ** (2 * r - 1)) == float(sp.factorial(2 * r - 1))


def test_generic_routine_is_the_pinned_za6_for_r3():
    rng = np.random.default_rng(0)
    for _ in range(300):
        f = rng.normal(size=6)
        f[rng.integers(0, 6):] += rng.normal() * 3
        assert oracle.za_flux(6, f) == oracle.za6_flux(f)


@pytest.mark.parametrize("order", [4, 8, 10])
def test_low_degree_polynomials_give_the_central_flux(order):
    rng = np.random.default_rng(order)
    r = order // 2
    c2r = oracle.coefficients_r(order)["c2r"]
    j = np.arange(2 * r, dtype=np.float64) - (r - 1)
    for _ in range(100):
        c = rng.integers(-20, 21, size=2 * r - 1).astype(np.float64)
        f = sum(c[k] * j ** k for k in range(2 * r - 1))
        scale = max(1.0, np.abs(f).max())
        assert abs(oracle.za_flux(order, f) - np.dot(c2r, f)) <= 1e-12 * scale


@pytest.mark.parametrize("order", [4, 8, 10])
def test_operator_order_on_smooth_data(order):
    r = order // 2
    errs = []
    for n in (5, 10, 20):
        dx = 1.0 / n
        xs = (np.arange(-r - 2, n + r + 3)) * dx
        fv = np.exp(2.0 * xs)
        def fh(jj):
            return oracle.za_flux(order, fv[jj + 3: jj + 2 * r + 3])
        errs.append(max(abs((fh(jj) - fh(jj - 1)) / dx - 2.0 * np.exp(2.0 * xs[jj + r + 2]))
                        for jj in range(n)))
    orders = [np.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert abs(orders[-1] - order) < 0.6, (errs, orders)


@pytest.mark.parametrize("order", [4, 8, 10])
def test_rhs_of_every_order_conserves(order):
    w = wl.smooth_euler_1d(n=64, seed=2)
    U = w["U"].copy()
    U[0, :, 0, 20:40] *= 1.2
    g = oracle.make_grid(ndim=1, nx=64, dx=w["dx"], bc_x="periodic", order=order)
    L = oracle.rhs(g, U)
    for k in range(3):
        assert abs(L[0, k].sum()) <= 1e-13 * np.abs(L[0, k]).sum()
    w = wl.burgers_sine(n=64)
    g = oracle.make_grid(system="burgers", ndim=1, nx=64, dx=w["dx"], bc_x="periodic", order=order)
    U2, _, _ = oracle.solve(g, w["U"], 0.5, 0.2)
    assert abs(U2.sum() - w["U"].sum()) <= 1e-13 * np.abs(w["U"]).sum()


@pytest.mark.parametrize("order", [4, 8, 10])
def test_sod_converges_for_every_order(order):
    errs = []
    for n in (200, 400):
        w = wl.shock_tube("sod", n=n)
        g = oracle.make_grid(ndim=1, nx=n, dx=w["dx"], order=order)
        U, _, _ = oracle.solve(g, w["U"], w["cfl"], w["t_final"])
        rho, _, _, _ = oracle.riemann_exact(w["left"], w["right"], w["x"], w["t_final"])
        errs.append(np.abs(U[0, 0, 0] - rho).mean())
    assert errs[1] < errs[0] < 0.02, errs

"""Pin the oracle's coefficient tables to their definitions (Section 2, Section 3).

Every table the oracle uses (c_6, c_k, d, B_k, c_tau) is re-derived here in
exact rational arithmetic from the defining equations, not from the printed
numbers: eqs. (8)-(9) (cell-average interpolation with dx = 1, x_i = 0),
eq. (12) (ideal weights), eq. (15) (smoothness indicators as scaled L2 norms
of the derivatives over I_i), and the consistency requirement on c_tau
(eq. (17): a (2r-1)-th derivative measure).
"""
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp

import oracle

X = sp.Symbol("x")


def _interp(nodes):
    """Polynomial of degree len(nodes)-1 whose averages over the unit cells
    centred at `nodes` equal symbols f_0..f_{m-1} (eq. (9), dx = 1)."""
    m = len(nodes)
    a = sp.symbols("a0:%d" % m)
    f = sp.symbols("f0:%d" % m)
    p = sum(a[n] * X ** n for n in range(m))
    eqs = [sp.integrate(p, (X, l - sp.Rational(1, 2), l + sp.Rational(1, 2))) - f[k]
           for k, l in enumerate(nodes)]
    sol = sp.solve(eqs, a, dict=True)[0]
    return sp.expand(p.subs(sol)), f


def _coeffs_at_half(nodes):
    p, f = _interp(nodes)
    val = sp.expand(p.subs(X, sp.Rational(1, 2)))
    return [sp.nsimplify(val.coeff(fk)) for fk in f]


def _frac(x, den=2000):
    return Fraction(x).limit_denominator(den)


@pytest.fixture(scope="module")
def tables():
    return oracle.coefficients()


def test_c6_from_interpolation(tables):
    # eq. (10): the central flux on S^6 = {x_{i-2}, ..., x_{i+3}}.
    want = _coeffs_at_half([-2, -1, 0, 1, 2, 3])
    got = [_frac(v) for v in tables["c6"]]
    assert [Fraction(int(w.p), int(w.q)) for w in want] == got


def test_ck_from_interpolation(tables):
    # eq. (11): S_k = {x_{i-2+k}, x_{i-1+k}, x_{i+k}}, k = 0..3.
    for k in range(4):
        want = _coeffs_at_half([k - 2, k - 1, k])
        got = [_frac(v) for v in tables["ck"][k]]
        assert [Fraction(int(w.p), int(w.q)) for w in want] == got, k


def test_ideal_weights_solve_linear_combination(tables):
    # eq. (12): sum_k d_k c_k (placed on S^6) = c_6; and d_k = C(3,k)^2 / C(6,3).
    c6 = _coeffs_at_half([-2, -1, 0, 1, 2, 3])
    d = sp.symbols("d0:4")
    rows = []
    for j in range(6):
        s = 0
        for k in range(4):
            if k <= j <= k + 2:
                s += d[k] * _coeffs_at_half([k - 2, k - 1, k])[j - k]
        rows.append(s - c6[j])
    sol = sp.solve(rows, d, dict=True)[0]
    want = [Fraction(int(sol[dk].p), int(sol[dk].q)) for dk in d]
    assert want == [Fraction(sp.binomial(3, k) ** 2, sp.binomial(6, 3)) for k in range(4)]
    assert [_frac(v) for v in tables["d"]] == want
    # the oracle's own tables satisfy the identity exactly in rationals
    ck = [[_frac(v) for v in row] for row in tables["ck"]]
    dd = [_frac(v) for v in tables["d"]]
    comb = [sum(dd[k] * ck[k][j - k] for k in range(4) if k <= j <= k + 2) for j in range(6)]
    assert comb == [_frac(v) for v in tables["c6"]]


def _beta_matrix(nodes):
    """eq. (15) with dx = 1, x_i = 0: beta = sum_{l=1}^{r-1} int_{-1/2}^{1/2} (p^(l))^2."""
    p, f = _interp(nodes)
    beta = 0
    for l in (1, 2):
        beta += sp.integrate(sp.diff(p, X, l) ** 2, (X, -sp.Rational(1, 2), sp.Rational(1, 2)))
    beta = sp.expand(beta)
    M = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            if a == b:
                M[a][b] = beta.coeff(f[a], 2)
            else:
                M[a][b] = beta.coeff(f[a], 1).coeff(f[b], 1) / 2
    return [[Fraction(int(sp.nsimplify(v).p), int(sp.nsimplify(v).q)) for v in row] for row in M]


@pytest.mark.parametrize("name,nodes", [("B0", [-2, -1, 0]), ("B1", [-1, 0, 1]),
                                        ("B2", [0, 1, 2]), ("Bd", [1, 2, 3])])
def test_smoothness_matrices_from_definition(tables, name, nodes):
    # B_d: the polynomial on the downwind substencil S_3, measured over I_i.
    want = _beta_matrix(nodes)
    got = [[_frac(v) for v in row] for row in tables[name]]
    assert got == want
    # B_k annihilates constants: the indicators see only the variation of f_k
    assert all(sum(row) == 0 for row in want)


def test_ctau_is_a_fifth_derivative_measure(tables):
    # eq. (17): <c_tau, f^6> annihilates polynomials of degree <= 4 and is
    # consistent with the 5th derivative: <c_tau, j^5> = 5! (dx = 1).
    c = tables["ctau"]
    j = np.arange(6, dtype=np.float64)
    for deg in range(5):
        assert np.dot(c, j ** deg) == 0.0
    assert np.dot(c, j ** 5) == 120.0

"""Pin the oracle's WENO-ZA6 operator to the paper's Tables 3 and 4 (Section 3.1).

The test function f = x^(ncp+1) exp(0.75 x) has a critical point of order
ncp at x = 0.  The oracle evaluates the operator (f_hat_{j+1/2} -
f_hat_{j-1/2}) / dx on the nodes of [-1, 1] and its L_inf error against f'.
Every printed error is matched to the two printed digits in quadruple
precision (the smallest entries lie below double rounding), every printed
order m to one decimal, and the double-precision oracle is matched on all
entries above 1e-10.  The ncp = 1 column is also checked against the closed
form of the linear sixth-order central difference error, |f^(7)| dx^6 / 140
at x = 1, which the weights approach there.
"""
import math
import os

import pytest
import sympy as sp

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")

# Two printed entries of Table 4 disagree with the printed convergence orders
# next to them (5.8E-14 and 2.3E-13 at 1/dx = 320 for ncp = 4, 5: the
# printed orders 6.0, 6.0 on either side require 5.6E-14 and 2.7E-13).  They
# are read as misprints; the orders around them are still checked.
MISPRINTS = {("table4", 320, 4), ("table4", 320, 5)}


def _read(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            inv_dx = int(t[0])
            vals = []
            for c in range(5):
                e = float(t[1 + 2 * c])
                m = None if t[2 + 2 * c] == "-" else float(t[2 + 2 * c])
                vals.append((e, m))
            rows.append((inv_dx, vals))
    return rows


def _params(table, ncp):
    if table == "table3":
        return 1.0, False
    return (1.5, False) if ncp <= 3 else (1.0, True)


@pytest.mark.parametrize("table,fname", [("table3", "table3_ncp_p1.txt"),
                                         ("table4", "table4_ncp_p15_vareps.txt")])
def test_printed_errors_and_orders_quad(table, fname):
    rows = _read(fname)
    for ncp in range(1, 6):
        p, var = _params(table, ncp)
        errs = []
        for inv_dx, vals in rows:
            e = oracle.operator_error(ncp, inv_dx, p=p, eps_variable=var, quad=True)
            errs.append(e)
            printed, m = vals[ncp - 1]
            if (table, inv_dx, ncp) not in MISPRINTS:
                assert "%.1E" % e == "%.1E" % printed, (table, ncp, inv_dx, e, printed)
            if m is not None:
                mine = math.log2(errs[-2] / errs[-1])
                assert abs(mine - m) <= 0.051, (table, ncp, inv_dx, mine, m)


def test_printed_errors_double():
    for inv_dx, vals in _read("table3_ncp_p1.txt"):
        for ncp in range(1, 6):
            printed = vals[ncp - 1][0]
            if printed < 1e-10:
                continue
            e = oracle.operator_error(ncp, inv_dx, p=1.0, quad=False)
            assert "%.1E" % e == "%.1E" % printed, (ncp, inv_dx, e)


def test_ncp1_column_is_linear_cd6_error():
    x = sp.Symbol("x")
    f7 = sp.diff(x ** 2 * sp.exp(sp.Rational(3, 4) * x), x, 7)
    f7_at_1 = float(abs(f7.subs(x, 1)))
    for inv_dx in (20, 40, 80, 160):
        closed = f7_at_1 / inv_dx ** 6 / 140.0
        e = oracle.operator_error(1, inv_dx, p=1.0, quad=True)
        assert abs(e / closed - 1.0) < 0.03, (inv_dx, e, closed)

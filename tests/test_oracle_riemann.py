"""Pin the oracle's exact Riemann solver by the jump conditions that define it.

The exact solution of a 1D Euler Riemann problem is fixed by gas dynamics:
across a shock the Rankine-Hugoniot conditions hold (mass, momentum and energy
fluxes continuous in the shock frame); across a rarefaction fan the entropy
p / rho^gamma and the outgoing Riemann invariant are constant; across the
contact p and u are continuous.  These are checked on the sampled profile of
each problem of the paper's shock-tube table (Section 4.2) and of a seeded
batch of random problems.
"""
import numpy as np
import pytest

import oracle
from paper_2603_26272_gb300 import workloads as wl

G = 1.4


def _E(r, u, p):
    return p / (G - 1) + 0.5 * r * u * u


def _check_wave(Wa, Wb, s, rtol=1e-9):
    """Rankine-Hugoniot between states a and b moving at speed s."""
    ra, ua, pa = Wa
    rb, ub, pb = Wb
    m_a, m_b = ra * (ua - s), rb * (ub - s)
    assert m_a == pytest.approx(m_b, rel=rtol, abs=1e-12)
    mom_a = ra * ua * (ua - s) + pa
    mom_b = rb * ub * (ub - s) + pb
    assert mom_a == pytest.approx(mom_b, rel=rtol, abs=1e-12)
    en_a = _E(ra, ua, pa) * (ua - s) + pa * ua
    en_b = _E(rb, ub, pb) * (ub - s) + pb * ub
    assert en_a == pytest.approx(en_b, rel=rtol, abs=1e-12)


def _verify(left, right, t=0.7):
    x = np.linspace(-20, 20, 400001)
    rho, u, p, star = oracle.riemann_exact(left, right, x, t)
    ps, us = star
    S = x / t
    # left wave
    rl, ul, pl = left
    rr, ur, pr = right
    left_star = (S < us) & (np.abs(p - ps) < 1e-12 * ps) & (np.abs(u - us) < 1e-12 * (1 + abs(us)))
    right_star = (S > us) & (np.abs(p - ps) < 1e-12 * ps) & (np.abs(u - us) < 1e-12 * (1 + abs(us)))
    assert left_star.any() and right_star.any()
    rsl = rho[left_star][0]
    rsr = rho[right_star][-1]
    # contact: pressure and velocity continuous by construction; densities differ
    if ps > pl:  # left shock
        s = (rsl * us - rl * ul) / (rsl - rl)
        _check_wave(left, (rsl, us, ps), s)
        # the profile jumps exactly at x = s t
        k = np.argmax(np.abs(np.diff(rho[(S < us)])))
        assert abs(x[k] - s * t) < 2 * (x[1] - x[0])
    else:  # left rarefaction: entropy and J+ = u + 2c/(g-1) constant
        fan = (S < us)
        c = np.sqrt(G * p[fan] / rho[fan])
        np.testing.assert_allclose(p[fan] / rho[fan] ** G, pl / rl ** G, rtol=1e-10)
        np.testing.assert_allclose(u[fan] + 2 * c / (G - 1), ul + 2 * np.sqrt(G * pl / rl) / (G - 1),
                                   rtol=1e-10, atol=1e-10)
    if ps > pr:  # right shock
        s = (rsr * us - rr * ur) / (rsr - rr)
        _check_wave((rsr, us, ps), right, s)
    else:
        fan = (S > us)
        c = np.sqrt(G * p[fan] / rho[fan])
        np.testing.assert_allclose(p[fan] / rho[fan] ** G, pr / rr ** G, rtol=1e-10)
        np.testing.assert_allclose(u[fan] - 2 * c / (G - 1), ur - 2 * np.sqrt(G * pr / rr) / (G - 1),
                                   rtol=1e-10, atol=1e-10)
    # far field untouched
    assert rho[0] == rl and rho[-1] == rr


@pytest.mark.parametrize("name", ["sod", "lax", "123"])
def test_paper_tubes_satisfy_jump_conditions(name):
    left, right, _ = wl.PAPER_TUBES[name]
    _verify(left, right)


def test_random_batch_satisfies_jump_conditions():
    w = wl.riemann_batch(nbatch=16, n=8, seed=2)
    for k in range(16):
        st = w["states"][k]
        _verify(tuple(st[0]), tuple(st[1]))


def test_symmetric_problems():
    # 123 problem: symmetric two-rarefaction solution, u* = 0 by symmetry.
    _, _, _, star = oracle.riemann_exact((1.0, -2.0, 0.4), (1.0, 2.0, 0.4), np.zeros(1), 1.0)
    assert abs(star[1]) < 1e-13
    # mirrored states give mirrored solutions
    x = np.linspace(-3, 3, 61)
    a = oracle.riemann_exact((0.125, 0.0, 0.1), (1.0, 0.0, 1.0), x, 1.0)
    b = oracle.riemann_exact((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), -x, 1.0)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12)
    np.testing.assert_allclose(a[1], -b[1], rtol=1e-12, atol=1e-14)

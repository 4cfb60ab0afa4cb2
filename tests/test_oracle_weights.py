"""Pin the oracle's nonlinear weights to what Sections 2.1-2.2 and 3 fix.

* Smooth data: a polynomial of degree <= 4 has tau = 0 (eq. (17)),
  so Gamma_k = 0 and the weights equal the ideal weights d: the flux is the
  linear central flux <c_6, f> of eq. (10) (Section 1, Section 3.1).
* Away from critical points omega_k - d_k falls much faster than dx^4
  (the sufficient condition eq. (28)).
* Near a discontinuity the weight ratio of eq. (23) falls like dx^(2p), and
  the downwind weight vanishes (Section 2.2).
* With Ai, the flux is affine invariant (eq. (22)): f_hat(a f + b) =
  a f_hat(f) + b; without it a tiny-amplitude jump loses adaptivity.
"""
import numpy as np
import pytest

import oracle

D = np.array([1, 9, 9, 1]) / 20.0
C6 = np.array([1, -8, 37, 37, -8, 1]) / 60.0


@pytest.mark.parametrize("ai", [0, 1])
def test_quartic_data_gives_linear_weights(ai):
    rng = np.random.default_rng(11)
    j = np.arange(6, dtype=np.float64) - 2.0
    for _ in range(200):
        c = rng.integers(-50, 51, size=5).astype(np.float64)
        f = c[0] + c[1] * j + c[2] * j ** 2 + c[3] * j ** 3 + c[4] * j ** 4  # exact integers
        r = oracle.za6_flux(f, ai=ai, detail=True)
        scale = max(1.0, np.abs(f).max())
        assert r["tau"] <= (1e-13 * scale) ** 2  # zero up to rounding of f - mean
        np.testing.assert_allclose(r["omega"], D, rtol=0, atol=1e-15)
        assert abs(r["fhat"] - np.dot(C6, f)) <= 1e-14 * scale


def test_quintic_has_nonzero_tau():
    j = np.arange(6, dtype=np.float64)
    r = oracle.za6_flux(j ** 5, detail=True)
    assert r["tau"] == 120.0 ** 2


def test_weights_are_convex():
    rng = np.random.default_rng(5)
    for _ in range(500):
        f = rng.normal(size=6) * 10 ** rng.uniform(-3, 3)
        if rng.random() < 0.5:
            f[rng.integers(1, 6):] += rng.normal() * 10
        for ai in (0, 1):
            r = oracle.za6_flux(f, ai=ai, detail=True)
            assert np.all(r["omega"] >= 0)
            assert abs(r["omega"].sum() - 1.0) < 1e-14


def test_smooth_weights_approach_ideal_fast():
    # f = exp(x) sampled with spacing h (no critical point): omega - d = O(h^8)
    # here, well inside the O(h^4) sufficient condition.
    devs = []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        f = np.exp(0.3 + h * (np.arange(6) - 2.0))
        r = oracle.za6_flux_quad(f)  # flux only
        rd = oracle.za6_flux(f, detail=True)
        devs.append(np.abs(rd["omega"] - D).max())
        assert abs(r - rd["fhat"]) < 1e-14
    for a, b in zip(devs, devs[1:]):
        assert np.log2(a / b) > 4.0


@pytest.mark.parametrize("p", [1.0, 2.0])
def test_discontinuous_substencil_suppressed_like_dx_2p(p):
    # Jump between stencil points 3 and 4: S_0, S_1 smooth, S_2 and S_d
    # discontinuous; S_3 is affected through the mean of eq. (16).
    ratios = []
    w3 = []
    for h in (0.04, 0.02, 0.01):
        x = 0.1 + h * (np.arange(6) - 2.0)
        f = np.sin(x) + np.where(np.arange(6) >= 4, 1.0, 0.0)
        r = oracle.za6_flux(f, p=p, detail=True)
        om = r["omega"]
        ratios.append((D[1] / D[2]) * om[2] / om[1])  # eq. (23), D = 2, S = 1
        w3.append(om[3])
    slopes = [np.log2(a / b) for a, b in zip(ratios, ratios[1:])]
    for s in slopes:
        assert abs(s - 2 * p) < 0.35, slopes
    assert w3[-1] < 1e-3 and w3[-1] < w3[0]


def test_downwind_ratio_bounds_eq24():
    # eq. (24): (d_r/d_D)(omega_D/omega_r) in (c^p, 1] with beta_r = c beta_D,
    # D the discontinuous substencil with the largest indicator.
    rng = np.random.default_rng(3)
    for _ in range(200):
        f = rng.normal(size=6) * 0.01
        f[rng.integers(2, 5):] += 1.0
        for p in (1.0, 1.5, 2.0):
            r = oracle.za6_flux(f, p=p, detail=True)
            beta = r["beta"]  # beta_0, beta_1, beta_2, beta_d, beta_3
            Dk = int(np.argmax(beta[:3]))
            if beta[Dk] < beta[3]:
                continue  # the premise 0 < c <= 1 needs beta_D >= beta_d
            c = beta[4] / beta[Dk]
            ratio = (D[3] / D[Dk]) * r["omega"][Dk] / r["omega"][3]
            assert c ** p - 1e-12 < ratio <= 1.0 + 1e-12


def test_affine_invariance_with_ai():
    rng = np.random.default_rng(7)
    for _ in range(300):
        f = rng.normal(size=6)
        if rng.random() < 0.5:
            f[rng.integers(1, 6):] += 3.0
        base = oracle.za6_flux(f, ai=1)
        for a in (1e-30, -2.5, 1e-6, 4e5):
            b = rng.normal() * 10
            got = oracle.za6_flux(a * f + b, ai=1)
            want = a * base + b
            assert abs(got - want) <= 1e-12 * (abs(a) * np.abs(f).max() + abs(b)), (a, got, want)


def test_tiny_jump_needs_ai():
    # A jump of amplitude 1e-25: without Ai, eps = 1e-40 dominates the tiny
    # indicators and the weights fall back to d (no adaptivity, eq. (21));
    # with Ai (eq. (22)) the weights and flux are those of the unit jump.
    f = np.where(np.arange(6) >= 3, 1.0, 0.0)
    unit = oracle.za6_flux(f, ai=1, detail=True)
    tiny_ai = oracle.za6_flux(1e-25 * f, ai=1, detail=True)
    tiny_no = oracle.za6_flux(1e-25 * f, ai=0, detail=True)
    np.testing.assert_allclose(tiny_ai["omega"], unit["omega"], rtol=0, atol=1e-14)
    assert abs(tiny_ai["fhat"] - 1e-25 * unit["fhat"]) <= 1e-12 * 1e-25
    np.testing.assert_allclose(tiny_no["omega"], D, rtol=1e-6)
    assert unit["omega"][0] > 1.0 - 1e-14


def test_constant_data_gives_constant_flux():
    for c in (0.0, 1.0, -3.7, 1e-200, 1e100):
        f = np.full(6, c)
        r = oracle.za6_flux(f, ai=1, detail=True)
        np.testing.assert_allclose(r["omega"], D, rtol=1e-15)
        assert r["fhat"] == pytest.approx(c, rel=1e-15, abs=0)


def test_quad_and_double_agree():
    rng = np.random.default_rng(9)
    for _ in range(200):
        f = rng.normal(size=6)
        f[rng.integers(0, 6):] += rng.normal() * 5
        for p in (1.0, 1.5, 2.0):
            a = oracle.za6_flux(f, p=p)
            b = oracle.za6_flux_quad(f, p=p)
            assert abs(a - b) <= 1e-13 * max(1.0, np.abs(f).max())


def test_flat_substencils_next_to_a_jump():
    # Flat substencils at a nonzero level beside a small jump: every beta_k
    # must be >= 0 (an integral of squares, eq. (15)) and exactly 0 where the
    # substencil is flat, and the flux must stay inside the data's range.
    rng = np.random.default_rng(13)
    for _ in range(2000):
        level = rng.uniform(-5, 5)
        f = np.full(6, level)
        k = rng.integers(1, 6)
        f[k:] += rng.normal() * 10 ** rng.uniform(-12, 0)
        r = oracle.za6_flux(f, ai=1, detail=True)
        assert np.all(r["beta"] >= 0)
        if k >= 3:
            assert r["beta"][0] == 0.0
        assert np.all(r["omega"] >= 0)
        lo, hi = f.min(), f.max()
        span = hi - lo
        assert lo - 1e-12 * span - 1e-15 * abs(level) <= r["fhat"] <= hi + 1e-12 * span + 1e-15 * abs(level)

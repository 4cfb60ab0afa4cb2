"""Symbolic check of the rewritten formulas the CUDA kernels evaluate.

The kernels (csrc/weno_device.cuh) do not evaluate the paper's formulas
literally; they use algebraically exact rewrites chosen for FP64 economy.
This test proves each rewrite equal to the paper's definition in exact
arithmetic (sympy).  It does not replace the GPU parity tests: it shows the
algebra is right, the parity tests show the code computes it.
"""
import sympy as sp

v = sp.symbols("v0:6")
d = [v[j + 1] - v[j] for j in range(5)]
s = [d[k + 1] - d[k] for k in range(4)]

# Section 3: printed smoothness matrices (eq. (15) for r = 3), B_2 = rev(B_0)
B0 = sp.Matrix([[8, -19, 11], [-19, 50, -31], [11, -31, 20]]) / 6
B1 = sp.Matrix([[8, -13, 5], [-13, 26, -13], [5, -13, 8]]) / 6
B2 = sp.Matrix(3, 3, lambda a, b: B0[2 - a, 2 - b])
Bd = sp.Matrix([[44, -73, 29], [-73, 122, -49], [29, -49, 20]]) / 6


def qf(B, f):
    f = sp.Matrix(f)
    return sp.expand((f.T * B * f)[0])


def test_difference_form_of_indicators():
    t = [3 * d[1] - d[0], d[1] + d[2], 3 * d[2] - d[3], 3 * d[4] - 5 * d[3]]
    four_beta = [sp.Rational(13, 3) * s[k] ** 2 + t[k] ** 2 for k in range(4)]
    paper = [qf(B0, v[0:3]), qf(B1, v[1:4]), qf(B2, v[2:5]), qf(Bd, v[3:6])]
    for k in range(4):
        assert sp.expand(four_beta[k] - 4 * paper[k]) == 0, k


def test_tau_as_difference_of_second_differences():
    ctau = [-1, 5, -10, 10, -5, 1]
    paper = sum(c * x for c, x in zip(ctau, v)) ** 2
    r5 = (s[3] - s[0]) + 3 * (s[1] - s[2])
    assert sp.expand(4 * r5 ** 2 - 4 * paper) == 0


def test_candidate_fluxes_as_corrections():
    ck = [(2, -7, 11), (-1, 5, 2), (2, 5, -1), (11, -7, 2)]
    r = [5 * d[1] - 2 * d[0], d[1] + 2 * d[2], 4 * d[2] - d[3], 6 * d[2] - 5 * d[3] + 2 * d[4]]
    for k in range(4):
        paper = sum(c * v[k + m] for m, c in enumerate(ck[k])) / 6
        assert sp.expand(v[2] + r[k] / 6 - paper) == 0, k


def test_mean_deviation_from_differences():
    a = [-(d[0] + d[1]), -d[1], 0, d[2], d[2] + d[3], d[2] + d[3] + d[4]]
    for j in range(6):
        assert sp.expand(a[j] - (v[j] - v[2])) == 0


def test_closed_form_left_eigenvectors_2d():
    un, ut, c, g = sp.symbols("u_n u_t c gamma", positive=True)
    q2 = un ** 2 + ut ** 2
    H = c ** 2 / (g - 1) + q2 / 2
    R = sp.Matrix([[1, 1, 0, 1],
                   [un - c, un, 0, un + c],
                   [ut, ut, 1, ut],
                   [H - un * c, q2 / 2, ut, H + un * c]])
    b1 = (g - 1) / c ** 2
    b2 = b1 * q2 / 2
    Lk = sp.Matrix([[(b2 + un / c) / 2, -(b1 * un + 1 / c) / 2, -b1 * ut / 2, b1 / 2],
                    [1 - b2, b1 * un, b1 * ut, -b1],
                    [-ut, 0, 1, 0],
                    [(b2 - un / c) / 2, -(b1 * un - 1 / c) / 2, -b1 * ut / 2, b1 / 2]])
    assert sp.simplify(Lk * R - sp.eye(4)) == sp.zeros(4, 4)
    # the kernel's projection with rows 2 l1, l2, l3, 2 l4
    rho, mn, mt, E = sp.symbols("rho m_n m_t E")
    sx = un * mn + ut * mt - E
    z = b2 * rho - b1 * sx
    tc = (un * rho - mn) / c
    kern = sp.Matrix([z + tc, rho - z, mt - ut * rho, z - tc])
    want = sp.diag(2, 1, 1, 2) * Lk * sp.Matrix([rho, mn, mt, E])
    assert sp.simplify(kern - want) == sp.zeros(4, 1)
    # back-projection of e = (h1/4, h2/2, h3/2, h4/4)
    h = sp.symbols("h1:5")
    e = [h[0] / 4, h[1] / 2, h[2] / 2, h[3] / 4]
    S = e[0] + e[3] + e[1]
    D = e[3] - e[0]
    F = sp.Matrix([S, un * S + c * D, ut * S + e[2], H * (e[0] + e[3]) + un * c * D + q2 / 2 * e[1] + ut * e[2]])
    assert sp.simplify(F - R * sp.Matrix(e)) == sp.zeros(4, 1)


def test_closed_form_left_eigenvectors_1d():
    u, c, g = sp.symbols("u c gamma", positive=True)
    H = c ** 2 / (g - 1) + u ** 2 / 2
    R = sp.Matrix([[1, 1, 1], [u - c, u, u + c], [H - u * c, u ** 2 / 2, H + u * c]])
    b1 = (g - 1) / c ** 2
    b2 = b1 * u ** 2 / 2
    rho, m, E = sp.symbols("rho m E")
    z = b2 * rho - b1 * (u * m - E)
    tc = (u * rho - m) / c
    kern = sp.Matrix([z + tc, rho - z, z - tc])
    want = sp.diag(2, 1, 2) * R.inv() * sp.Matrix([rho, m, E])
    assert sp.simplify(kern - want) == sp.zeros(3, 1)


def test_division_free_weights():
    # omega_k = d_k (1 + T/b_k) / sum_j d_j (1 + T/b_j)
    #         = d_k (b_k + T) prod_{j!=k} b_j / sum_j d_j (b_j + T) prod_{i!=j} b_i,
    # and an exact common scale of b and T leaves it unchanged.
    b = sp.symbols("b0:4", positive=True)
    T, sc = sp.symbols("T sc", positive=True)
    dk = [1, 9, 9, 1]
    paper = [dk[k] * (1 + T / b[k]) for k in range(4)]
    bs = [sc * x for x in b]
    Ts = sc * T
    kern = [dk[0] * (bs[0] + Ts) * (bs[1] * (bs[2] * bs[3])),
            (bs[1] + Ts) * (9 * (bs[0] * (bs[2] * bs[3]))),
            (bs[2] + Ts) * (9 * (bs[3] * (bs[0] * bs[1]))),
            (bs[3] + Ts) * (bs[2] * (bs[0] * bs[1]))]
    for k in range(4):
        assert sp.simplify(paper[k] / sum(paper) - kern[k] / sum(kern)) == 0


def test_candidate_corrections_share_the_indicator_terms():
    # r0 = 5d1 - 2d0 = 2 t0 - d1 and r3 = 6d2 - 5d3 + 2d4 = 6d2 + (t3 - d4)
    t0 = 3 * d[1] - d[0]
    t3 = 3 * d[4] - 5 * d[3]
    assert sp.expand((2 * t0 - d[1]) - (5 * d[1] - 2 * d[0])) == 0
    assert sp.expand((6 * d[2] + (t3 - d[4])) - (6 * d[2] - 5 * d[3] + 2 * d[4])) == 0


def test_partial_sums_and_pair_flux():
    # za6 returns v2, num = sum a_k r_k (with d_1/d_0 = 9 applied as
    # 9 (a1 r1 + a2 r2)), den = a0 + a3 + 9 (a1 + a2); the flux is
    # v2 + num / (6 den); pair_flux adds two of them with one division.
    a = sp.symbols("a0:4", positive=True)
    r = sp.symbols("r0:4")
    v2p, v2m = sp.symbols("v2p v2m")
    num = 9 * (a[1] * r[1] + a[2] * r[2]) + (a[0] * r[0] + a[3] * r[3])
    den = 9 * (a[1] + a[2]) + (a[0] + a[3])
    w = [a[0], 9 * a[1], 9 * a[2], a[3]]
    want = v2p + sum(w[k] * r[k] / 6 for k in range(4)) / sum(w)
    assert sp.simplify(v2p + num / (6 * den) - want) == 0
    np_, dp, nm, dm = sp.symbols("n_p d_p n_m d_m", positive=True)
    pair = (v2p + v2m) + (np_ * dm + nm * dp) / (dp * dm) / 6
    assert sp.simplify(pair - (v2p + np_ / (6 * dp) + v2m + nm / (6 * dm))) == 0


def test_flux_projection_from_state_projection():
    # F = u_n U + p (0, 1, 0, u_n) in the normal frame (eq. (25)), so the
    # characteristic values of F follow from those of U, u_n and p.
    un, ut, c, g = sp.symbols("u_n u_t c gamma", positive=True)
    q2 = un ** 2 + ut ** 2
    b1 = (g - 1) / c ** 2
    b2 = b1 * q2 / 2

    def project4(rho, mn, mt, E):
        sx = un * mn + ut * mt - E
        z = b2 * rho - b1 * sx
        tc = (un * rho - mn) / c
        return sp.Matrix([z + tc, rho - z, mt - ut * rho, z - tc])

    rho, uj, vt, p = sp.symbols("rho u_j v_t p", positive=True)
    mn, mt = rho * uj, rho * vt
    E = p / (g - 1) + rho * (uj ** 2 + vt ** 2) / 2
    F = [mn, mn * uj + p, mt * uj, (E + p) * uj]
    w = project4(rho, mn, mt, E)
    z = b1 * (uj - un)
    kern = sp.Matrix([uj * w[0] + (p * z - p / c), uj * w[1] - p * z, uj * w[2],
                      uj * w[3] + (p * z + p / c)])
    assert sp.simplify(kern - project4(*F)) == sp.zeros(4, 1)


def test_weights_as_product_plus_tau_times_cofactor():
    # a_k = (b_k + T) prod_{j != k} b_j = P + T Q_k, P = prod_j b_j, Q_k = P / b_k
    b = sp.symbols("b0:4", positive=True)
    T = sp.symbols("T", positive=True)
    P = b[0] * b[1] * b[2] * b[3]
    Q = [b[1] * (b[2] * b[3]), b[0] * (b[2] * b[3]), b[3] * (b[0] * b[1]), b[2] * (b[0] * b[1])]
    for k in range(4):
        assert sp.expand((b[k] + T) * Q[k] - (P + T * Q[k])) == 0


def test_backprojection_returns_four_times_the_flux():
    un, ut, c, g = sp.symbols("u_n u_t c gamma", positive=True)
    q2 = un ** 2 + ut ** 2
    H = c ** 2 / (g - 1) + q2 / 2
    R = sp.Matrix([[1, 1, 0, 1],
                   [un - c, un, 0, un + c],
                   [ut, ut, 1, ut],
                   [H - un * c, q2 / 2, ut, H + un * c]])
    h = sp.symbols("h1:5")
    e = sp.Matrix([h[0] / 4, h[1] / 2, h[2] / 2, h[3] / 4])
    h14 = h[0] + h[3]
    S = 2 * h[1] + h14
    D = h[3] - h[0]
    h3x2 = 2 * h[2]
    kern = sp.Matrix([S, un * S + c * D, ut * S + h3x2,
                      H * h14 + un * c * D + q2 * h[1] + ut * h3x2])
    assert sp.simplify(kern - 4 * R * e) == sp.zeros(4, 1)
    # 1D
    u = sp.symbols("u")
    H1 = c ** 2 / (g - 1) + u ** 2 / 2
    R1 = sp.Matrix([[1, 1, 1], [u - c, u, u + c], [H1 - u * c, u ** 2 / 2, H1 + u * c]])
    e1 = sp.Matrix([h[0] / 4, h[1] / 2, h[2] / 4])
    h13 = h[0] + h[2]
    S1 = 2 * h[1] + h13
    D1 = h[2] - h[0]
    kern1 = sp.Matrix([S1, u * S1 + c * D1, H1 * h13 + u * c * D1 + u ** 2 * h[1]])
    assert sp.simplify(kern1 - 4 * R1 * e1) == sp.zeros(3, 1)


def test_split_applied_to_differences():
    # f+ = g + A w on (i-2 .. i+3); f- = g - A w read from i+3 down to i-2
    w = sp.symbols("w0:6")
    g = sp.symbols("g0:6")
    A = sp.symbols("A")
    fp = [g[j] + A * w[j] for j in range(6)]
    fm = [g[5 - j] - A * w[5 - j] for j in range(6)]  # mirrored stencil
    dw = [w[j + 1] - w[j] for j in range(5)]
    dg = [g[j + 1] - g[j] for j in range(5)]
    dp = [A * dw[j] + dg[j] for j in range(5)]
    dm = [None] * 5
    for j in range(5):
        dm[4 - j] = A * dw[j] - dg[j]
    for j in range(5):
        assert sp.expand(dp[j] - (fp[j + 1] - fp[j])) == 0
        assert sp.expand(dm[j] - (fm[j + 1] - fm[j])) == 0
    base = -A * dw[2] + (g[2] + g[3])
    assert sp.expand(base - (fp[2] + fm[2])) == 0


def test_cubic_newton_reciprocal_step():
    # r1 = r0 + r0 (e + e^2), e = 1 - x r0  =>  1 - x r1 = e^3: a seed within
    # 2^-22 of 1/x gives 1/x to 2^-66 before the final roundings
    x, r0 = sp.symbols("x r0", positive=True)
    e = 1 - x * r0
    r1 = r0 + r0 * (e + e ** 2)
    assert sp.expand((1 - x * r1) - e ** 3) == 0


def test_pairwise_weight_products():
    # za6d forms a_k = (b_k + T) prod_{j != k} b_j pairwise: with p01 = b0 b1,
    # p23 = b2 b3, x0 = p01 + T b1, y1 = 9 (p01 + T b0), y2 = 9 (p23 + T b3),
    # x3 = p23 + T b2, num = p23 (y1 r1 + x0 r0) + p01 (y2 r2 + x3 r3) and
    # den = p23 (x0 + y1) + p01 (y2 + x3) are sum d_k a_k r_k and sum d_k a_k
    # with the linear weights d = (1, 9, 9, 1) (times 20).
    b = sp.symbols("b0:4", positive=True)
    r = sp.symbols("r0:4")
    T = sp.symbols("T", positive=True)
    dk = [1, 9, 9, 1]
    a = [(b[k] + T) * sp.prod([b[j] for j in range(4) if j != k]) for k in range(4)]
    p01, p23 = b[0] * b[1], b[2] * b[3]
    x0, y1 = p01 + T * b[1], 9 * (p01 + T * b[0])
    y2, x3 = 9 * (p23 + T * b[3]), p23 + T * b[2]
    num = p23 * (y1 * r[1] + x0 * r[0]) + p01 * (y2 * r[2] + x3 * r[3])
    den = p23 * (x0 + y1) + p01 * (y2 + x3)
    assert sp.expand(num - sum(dk[k] * a[k] * r[k] for k in range(4))) == 0
    assert sp.expand(den - sum(dk[k] * a[k] for k in range(4))) == 0


def test_centre_values_back_project_to_the_physical_flux():
    # The 2D sixth-order kernel reconstructs from differences only and leaves
    # out the centre values g_i + g_{i+1} = P(F_i + F_{i+1}) of every field
    # (P: project4, the scaled left eigenvectors 2 l1, l2, l3, 2 l4).  Their
    # back-projection R (c1, 2 c2, 2 c3, c4) is 2 (F_i + F_{i+1}) for any
    # F_i + F_{i+1} (R L = I), which the kernel adds as 4 F_i + 2 (F_{i+1} - F_i).
    un, ut, c, g = sp.symbols("u_n u_t c gamma", positive=True)
    q2 = un ** 2 + ut ** 2
    H = c ** 2 / (g - 1) + q2 / 2
    b1 = (g - 1) / c ** 2
    b2 = b1 * q2 / 2

    def project4(rho, mn, mt, E):
        sx = un * mn + ut * mt - E
        z = b2 * rho - b1 * sx
        tc = (un * rho - mn) / c
        return [z + tc, rho - z, mt - ut * rho, z - tc]

    def backproject4(h1, h2, h3, h4):
        h14 = h1 + h4
        S = 2 * h2 + h14
        D = h4 - h1
        return sp.Matrix([S, un * S + c * D, ut * S + 2 * h3,
                          H * h14 + un * c * D + q2 * h2 + ut * 2 * h3])

    FL = sp.symbols("FL0:4")
    dF = sp.symbols("dF0:4")
    FR = [FL[q] + dF[q] for q in range(4)]
    cvals = [x + y for x, y in zip(project4(*FL), project4(*FR))]
    kern = sp.Matrix([4 * FL[q] + 2 * dF[q] for q in range(4)])
    assert sp.simplify(backproject4(*cvals) - kern) == sp.zeros(4, 1)
    # the projection is linear: the differences of projected states are the
    # projected differences (what the kernel projects)
    U0, U1 = sp.symbols("a0:4"), sp.symbols("c0:4")
    lhs = [y - x for x, y in zip(project4(*U0), project4(*U1))]
    rhs = project4(*[U1[q] - U0[q] for q in range(4)])
    assert all(sp.expand(x - y) == 0 for x, y in zip(lhs, rhs))


def test_normal_flux_from_staged_values():
    # the kernel stages u_n and H = (E + p) / rho and forms p = rho H - E,
    # F1 = m_n u_n + p, F2 = m_t u_n, F3 = H m_n (eq. (25) in the normal frame)
    rho, un, ut, p, g = sp.symbols("rho u_n u_t p gamma", positive=True)
    mn, mt = rho * un, rho * ut
    E = p / (g - 1) + rho * (un ** 2 + ut ** 2) / 2
    H = (E + p) / rho
    assert sp.simplify(rho * H - E - p) == 0
    assert sp.simplify(H * mn - (E + p) * un) == 0


def test_third_order_reciprocal_square_root_step():
    # r1 = r (1 + e/2 + 3 e^2 / 8), e = 1 - x r^2: the series of (1 - e)^(-1/2)
    # to second order, so r1 sqrt(x) = 1 - (5/16) e^3 + O(e^4): a seed within
    # 2^-22 gives 1/sqrt(x) to about 2^-64 before the final roundings
    e = sp.symbols("e")
    # r sqrt(x) = (1 - e)^(1/2) exactly
    r1_sqrtx = sp.sqrt(1 - e) * (1 + e / 2 + sp.Rational(3, 8) * e ** 2)
    ser = sp.series(r1_sqrtx, e, 0, 4).removeO()
    assert sp.expand(ser - (1 - sp.Rational(5, 16) * e ** 3)) == 0

"""Pins of the oracle's characteristic decomposition (Section 4.2) and of its
global Lax-Friedrichs speeds (eq. (6)) against what the mathematics fixes.

The paper splits the Euler fluxes characteristic-wise on the Roe-averaged
state but prints no eigen-system.  Its parts are fixed independently of the
oracle's own formulas:
  * the flux Jacobian A(U) = dF/dU is taken here by complex-step
    differentiation of the Euler flux written out below (exact to rounding),
    so R must satisfy A R = R diag(lam) at the Roe state and L R = I;
  * the Roe average is the one state whose Jacobian satisfies
    F(U_R) - F(U_L) = A(U_roe) (U_R - U_L) (Roe's property); an arithmetic
    face average fails it;
  * the GLF speed of field m is the largest |lambda_m| of A over the cells of
    the stage input, in both directions, with the eigenvalues of A computed
    here by numpy from the complex-step Jacobian.
"""
import numpy as np
import pytest

import oracle

GAMMA = 1.4


def euler_flux(U, dir, gamma=GAMMA):
    """Physical flux of the Euler equations (eq. (25) and its 2D form) in
    direction dir, for real or complex conserved states (rho, m[, n], E)."""
    U = np.asarray(U)
    if U.size == 3:
        rho, m, E = U
        u = m / rho
        p = (gamma - 1.0) * (E - 0.5 * m * u)
        return np.array([m, m * u + p, (E + p) * u])
    rho, mx, my, E = U
    u, v = mx / rho, my / rho
    p = (gamma - 1.0) * (E - 0.5 * (mx * u + my * v))
    un = u if dir == 0 else v
    return np.array([rho * un, mx * un + (p if dir == 0 else 0.0),
                     my * un + (p if dir == 1 else 0.0), (E + p) * un])


def jacobian(U, dir, gamma=GAMMA, h=1e-30):
    """dF/dU by the complex step: Im F(U + i h e_k) / h (no cancellation)."""
    U = np.asarray(U, dtype=np.complex128)
    n = U.size
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1j * h
        A[:, k] = euler_flux(U + e, dir, gamma).imag / h
    return A


def conserved_from(rho, u, v, H, nc, gamma=GAMMA):
    """A conserved state with velocity (u, v) and total enthalpy H."""
    q2 = u * u + (v * v if nc == 4 else 0.0)
    p = rho * (gamma - 1.0) / gamma * (H - 0.5 * q2)
    E = p / (gamma - 1.0) + 0.5 * rho * q2
    if nc == 3:
        return np.array([rho, rho * u, E])
    return np.array([rho, rho * u, rho * v, E])


def random_state(rng, nc):
    rho = rng.uniform(0.1, 3.0)
    u = rng.uniform(-2.0, 2.0)
    v = rng.uniform(-2.0, 2.0) if nc == 4 else 0.0
    p = rng.uniform(0.05, 5.0)
    E = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.array([rho, rho * u, E]) if nc == 3 else np.array([rho, rho * u, rho * v, E])


CASES = [(3, 0), (4, 0), (4, 1)]


@pytest.mark.parametrize("nc,dir", CASES)
def test_roe_property(nc, dir):
    """R diag(lam) L (U_R - U_L) = F(U_R) - F(U_L): the face state is Roe's
    average and (R, lam, L) is the eigen-system of A there."""
    rng = np.random.default_rng(10 + 3 * nc + dir)
    for _ in range(200):
        UL, UR = random_state(rng, nc), random_state(rng, nc)
        f = oracle.roe_face(UL, UR, dir=dir)
        lhs = f["R"] @ np.diag(f["lam"]) @ f["L"] @ (UR - UL)
        rhs = euler_flux(UR, dir) - euler_flux(UL, dir)
        scale = np.abs(euler_flux(UR, dir)).max() + np.abs(euler_flux(UL, dir)).max()
        assert np.abs(lhs - rhs).max() <= 1e-13 * scale


@pytest.mark.parametrize("nc,dir", CASES)
def test_roe_property_fails_for_an_arithmetic_average(nc, dir):
    """Control: the Jacobian at the arithmetic mean of the primitive states
    does not satisfy Roe's property, so the test above can tell them apart."""
    rng = np.random.default_rng(77)
    worst = 0.0
    for _ in range(50):
        UL, UR = random_state(rng, nc), random_state(rng, nc)
        Um = 0.5 * (UL + UR)
        rhs = euler_flux(UR, dir) - euler_flux(UL, dir)
        lhs = jacobian(Um, dir) @ (UR - UL)
        worst = max(worst, np.abs(lhs - rhs).max() / np.abs(rhs).max())
    assert worst > 1e-3


@pytest.mark.parametrize("nc,dir", CASES)
def test_eigenpairs_of_the_flux_jacobian(nc, dir):
    """A(U_roe) R = R diag(lam) and L R = I at the Roe state, with A taken
    independently (complex step of the flux above)."""
    rng = np.random.default_rng(20 + 3 * nc + dir)
    for _ in range(100):
        UL, UR = random_state(rng, nc), random_state(rng, nc)
        f = oracle.roe_face(UL, UR, dir=dir)
        Uroe = conserved_from(1.7, f["u"], f["v"], f["H"], nc)
        A = jacobian(Uroe, dir)
        R, L, lam = f["R"], f["L"], f["lam"]
        s = np.abs(A).max() * np.abs(R).max()
        assert np.abs(A @ R - R @ np.diag(lam)).max() <= 1e-13 * s
        assert np.abs(L @ R - np.eye(nc)).max() <= 1e-13 * np.abs(L).max() * np.abs(R).max()
        # the eigenvalues are those of A, in ascending order u-c, u, (u), u+c
        ev = np.sort(np.linalg.eigvals(A).real)
        assert np.allclose(lam, ev, rtol=0, atol=1e-12 * (abs(f["u"]) + abs(f["v"]) + f["c"]))
        # c is the sound speed of the Roe state: c^2 = (gamma - 1)(H - q^2/2)
        q2 = f["u"] ** 2 + f["v"] ** 2
        assert f["c"] == pytest.approx(np.sqrt((GAMMA - 1) * (f["H"] - 0.5 * q2)), rel=1e-14)


def test_roe_face_of_equal_states_is_the_cell_state():
    rng = np.random.default_rng(3)
    U = random_state(rng, 4)
    f = oracle.roe_face(U, U, dir=0)
    rho = U[0]
    assert f["u"] == pytest.approx(U[1] / rho, rel=1e-15)
    assert f["v"] == pytest.approx(U[2] / rho, rel=1e-15)
    p = (GAMMA - 1) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
    assert f["H"] == pytest.approx((U[3] + p) / rho, rel=1e-14)


def test_roe_face_rejects_nonphysical_states():
    with pytest.raises(oracle.OracleError):
        oracle.roe_face(np.array([-1.0, 0.0, 1.0]), np.array([1.0, 0.0, 1.0]))


def _two_state_grid(rng, ndim, alpha_mode):
    nc = 3 if ndim == 1 else 4
    nx, ny = (7, 1) if ndim == 1 else (5, 4)
    A, B = random_state(rng, nc), random_state(rng, nc)
    U = np.empty((1, nc, ny, nx))
    mask = rng.random((ny, nx)) < 0.5
    mask.flat[0], mask.flat[1] = True, False  # both states present
    for k in range(nc):
        U[0, k] = np.where(mask, A[k], B[k])
    g = oracle.make_grid(ndim=ndim, nx=nx, ny=ny, alpha_mode=alpha_mode)
    return g, U, (A, B)


@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("alpha_mode", ["field", "single"])
def test_glf_speeds_are_jacobian_eigenvalue_maxima(ndim, alpha_mode):
    """Eq. (6): alpha of field m and direction dir = max over the cells of
    |lambda_m(A_dir(U))|, the eigenvalues of the Jacobian in ascending order
    (u-c, u, [u], u+c); alpha_mode 'single' = the largest over all fields."""
    rng = np.random.default_rng(40 + ndim)
    for _ in range(20):
        g, U, states = _two_state_grid(rng, ndim, alpha_mode)
        nc = U.shape[1]
        al = oracle.alpha(g, U)[0]
        for dir in range(ndim):
            want = np.zeros(nc)
            for S in states:
                ev = np.sort(np.linalg.eigvals(jacobian(S, dir)).real)
                want = np.maximum(want, np.abs(ev))
            if alpha_mode == "single":
                want[:] = want.max()
            assert np.allclose(al[dir, :nc], want, rtol=1e-12, atol=0)
            assert np.all(al[dir, nc:] == 0.0)
        if ndim == 1:
            assert np.all(al[1] == 0.0)

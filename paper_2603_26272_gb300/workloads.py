"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no WENO arithmetic: it only lays out initial conditions on
uniform grids, so that the CUDA path and the CPU oracle can be fed the same
bytes.  Conserved variables are formed from primitive ones with the ideal-gas
relation E = p/(gamma-1) + rho |u|^2 / 2 (Section 4.2, the equation of state
below eq. (25)).

Layout of every state: numpy float64 array [nbatch][ncomp][ny][nx], x fastest;
ncomp = 1 (advection), 3 (1D Euler: rho, rho u, E), 4 (2D Euler: rho, rho u,
rho v, E).  Cell centres are x_i = a + (i + 1/2) dx, i = 0 .. n-1.

Each generator returns a dict with the state "U" and the problem parameters
("domain", "n", "bc", "gamma", "cfl", "t_final" and so on).
"""
import numpy as np

GAMMA = 1.4


def cell_centres(a, b, n):
    dx = (b - a) / n
    return a + (np.arange(n) + 0.5) * dx, dx


def cons_1d(rho, u, p, gamma=GAMMA):
    rho, u, p = np.broadcast_arrays(np.asarray(rho, float), np.asarray(u, float),
                                    np.asarray(p, float))
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def cons_2d(rho, u, v, p, gamma=GAMMA):
    rho, u, v, p = np.broadcast_arrays(*(np.asarray(a, float) for a in (rho, u, v, p)))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def advection_sine(n=200, cfl=0.5, t_final=2.0):
    """u_t + u_x = 0 on periodic [-1, 1], u0 = sin(pi x - sin(pi x)/pi)."""
    x, dx = cell_centres(-1.0, 1.0, n)
    u0 = np.sin(np.pi * x - np.sin(np.pi * x) / np.pi)
    return {"system": "advection", "ndim": 1, "U": u0.reshape(1, 1, 1, n), "x": x, "dx": dx,
            "domain": (-1.0, 1.0), "n": n, "bc": "periodic", "cfl": cfl, "t_final": t_final,
            "exact": lambda xx, t: np.sin(np.pi * (xx - t) - np.sin(np.pi * (xx - t)) / np.pi)}


def burgers_sine(n=80, t_final=0.2, cfl=0.5):
    """Burgers u_t + (u^2/2)_x = 0 with u0 = 1/2 + sin(2 pi x) (Section 4.1,
    Table 5: N = 80, T = 0.2); reading: periodic [0, 1], one period of u0."""
    x, dx = cell_centres(0.0, 1.0, n)
    return {"system": "burgers", "ndim": 1, "U": (0.5 + np.sin(2 * np.pi * x)).reshape(1, 1, 1, n),
            "x": x, "dx": dx, "domain": (0.0, 1.0), "n": n, "bc": "periodic", "cfl": cfl,
            "t_final": t_final}


def buckley_leverett(n=200, t_final=0.3, cfl=0.5, a=-1.0, b=1.0):
    """Buckley-Leverett with u0 = 1 on [-0.5, 0], 0 elsewhere (Section 4.1,
    Table 5: N = 200, T = 0.3); reading: transmissive [-1, 1]."""
    x, dx = cell_centres(a, b, n)
    u0 = np.where((x >= -0.5) & (x <= 0.0), 1.0, 0.0)
    return {"system": "buckley_leverett", "ndim": 1, "U": u0.reshape(1, 1, 1, n), "x": x, "dx": dx,
            "domain": (a, b), "n": n, "bc": "transmissive", "cfl": cfl, "t_final": t_final}


def buckley_riemann(n=400, t_final=0.3, cfl=0.5, a=-1.0, b=1.0):
    """Buckley-Leverett Riemann problem u = 1 for x < 0, u = 0 for x > 0."""
    x, dx = cell_centres(a, b, n)
    return {"system": "buckley_leverett", "ndim": 1, "U": np.where(x < 0, 1.0, 0.0).reshape(1, 1, 1, n),
            "x": x, "dx": dx, "domain": (a, b), "n": n, "bc": "transmissive", "cfl": cfl,
            "t_final": t_final}


def shock_density(n=1600, a=-5.0, b=5.0, t_final=1.8, cfl=0.5, gamma=GAMMA):
    """Mach-3 shock meeting a density wave (Section 4.2, shock-density example):
    (3.857143, 2.629369, 10.33333) for x < -4, (1 + 0.2 sin 5x, 0, 1) beyond."""
    x, dx = cell_centres(a, b, n)
    left = x < -4.0
    rho = np.where(left, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
    u = np.where(left, 2.629369, 0.0)
    p = np.where(left, 10.33333, 1.0)
    U = cons_1d(rho, u, p, gamma).reshape(1, 3, 1, n)
    return {"system": "euler", "ndim": 1, "U": U, "x": x, "dx": dx, "domain": (a, b), "n": n,
            "bc": "transmissive", "cfl": cfl, "t_final": t_final, "gamma": gamma}


PAPER_TUBES = {  # Section 4.2, Riemann problems table: (left), (right), T
    "sod": ((0.125, 0.0, 0.1), (1.0, 0.0, 1.0), 2.0),
    "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 1.3),
    "123": ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4), 1.0),
}


def shock_tube(name, n=200, a=-5.0, b=5.0, x0=0.0, cfl=0.45, gamma=GAMMA):
    """The paper's shock tubes on [-5, 5] with the jump at 0 and its CFL 0.45
    (Section 4 preamble); at CFL 0.5 the near-vacuum of the 123 problem drives
    the unlimited scheme to a negative pressure."""
    left, right, T = PAPER_TUBES[name]
    return riemann_1d(left, right, x0=x0, n=n, a=a, b=b, t_final=T, cfl=cfl, gamma=gamma)


def riemann_1d(left, right, x0=0.0, n=200, a=-5.0, b=5.0, t_final=1.0, cfl=0.5, gamma=GAMMA):
    x, dx = cell_centres(a, b, n)
    L = x < x0
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    return {"system": "euler", "ndim": 1, "U": cons_1d(rho, u, p, gamma).reshape(1, 3, 1, n),
            "x": x, "dx": dx, "domain": (a, b), "n": n, "bc": "transmissive", "cfl": cfl,
            "t_final": t_final, "gamma": gamma, "left": tuple(left), "right": tuple(right),
            "x0": x0}


def riemann_batch(nbatch=64, n=1600, seed=2, a=-5.0, b=5.0, t_final=0.4, cfl=0.5, gamma=GAMMA):
    """Seeded batch of 1D Riemann problems: rho, p ~ U[0.1, 2], u ~ U[-1, 1]
    on each side, jump at x0 ~ U[-2, 2], transmissive ends."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 2.0, size=(nbatch, 2))
    u = rng.uniform(-1.0, 1.0, size=(nbatch, 2))
    p = rng.uniform(0.1, 2.0, size=(nbatch, 2))
    x0 = rng.uniform(-2.0, 2.0, size=nbatch)
    x, dx = cell_centres(a, b, n)
    U = np.empty((nbatch, 3, 1, n))
    for k in range(nbatch):
        L = x < x0[k]
        U[k, :, 0, :] = cons_1d(np.where(L, rho[k, 0], rho[k, 1]), np.where(L, u[k, 0], u[k, 1]),
                                np.where(L, p[k, 0], p[k, 1]), gamma)
    return {"system": "euler", "ndim": 1, "U": U, "x": x, "dx": dx, "domain": (a, b), "n": n,
            "bc": "transmissive", "cfl": cfl, "t_final": t_final, "gamma": gamma,
            "states": np.stack([rho, u, p], axis=-1), "x0": x0, "nbatch": nbatch}


def _quadrants(n, line, states, gamma, domain=(0.0, 1.0)):
    x, dx = cell_centres(domain[0], domain[1], n)
    X = x[None, :]
    Y = x[:, None]
    q = np.where(X > line, np.where(Y > line, 0, 3), np.where(Y > line, 1, 2))  # [ny][nx]
    rho = states[q, 0]
    u = states[q, 1]
    v = states[q, 2]
    p = states[q, 3]
    return cons_2d(rho, u, v, p, gamma).reshape(1, 4, n, n), dx


def quadrant_2d(n=2048, seed=3, line=0.5, steps=200, cfl=0.5, gamma=GAMMA):
    """Four-quadrant 2D Riemann data on [0,1]^2 with seeded states
    rho, p ~ U[0.1, 1.5], u, v ~ U[-1, 1]; quadrants numbered
    0: x>l, y>l; 1: x<l, y>l; 2: x<l, y<l; 3: x>l, y<l."""
    rng = np.random.default_rng(seed)
    st = np.empty((4, 4))
    st[:, 0] = rng.uniform(0.1, 1.5, 4)
    st[:, 1] = rng.uniform(-1.0, 1.0, 4)
    st[:, 2] = rng.uniform(-1.0, 1.0, 4)
    st[:, 3] = rng.uniform(0.1, 1.5, 4)
    U, dx = _quadrants(n, line, st, gamma)
    return {"system": "euler", "ndim": 2, "U": U, "dx": dx, "dy": dx, "domain": (0.0, 1.0),
            "n": n, "bc": "transmissive", "cfl": cfl, "steps": steps, "gamma": gamma,
            "states": st}


def config3_2d(n=400, cfl=0.45, t_final=0.8, gamma=GAMMA):
    """Configuration 3 of the 2D Riemann problem (Section 4.3), lines at 0.8."""
    st = np.array([[1.5, 0.0, 0.0, 1.5],
                   [0.5323, 1.206, 0.0, 0.3],
                   [0.138, 1.206, 1.206, 0.029],
                   [0.5323, 0.0, 1.206, 0.3]])
    U, dx = _quadrants(n, 0.8, st, gamma)
    return {"system": "euler", "ndim": 2, "U": U, "dx": dx, "dy": dx, "domain": (0.0, 1.0),
            "n": n, "bc": "transmissive", "cfl": cfl, "t_final": t_final, "gamma": gamma,
            "states": st}


def smooth_euler_1d(n=64, seed=0, a=0.0, b=1.0, gamma=GAMMA, amp=0.2):
    """Smooth periodic 1D Euler data (random low Fourier modes), for
    conservation and symmetry checks."""
    rng = np.random.default_rng(seed)
    x, dx = cell_centres(a, b, n)
    k = np.arange(1, 4)
    def field(base, s):
        c = rng.normal(size=(3, 2)) * s
        return base + (c[:, :1] * np.sin(2 * np.pi * k[:, None] * x) +
                       c[:, 1:] * np.cos(2 * np.pi * k[:, None] * x)).sum(0)
    rho = field(1.0, amp)
    u = field(0.3, amp)
    p = field(1.0, amp)
    return {"system": "euler", "ndim": 1, "U": cons_1d(rho, u, p, gamma).reshape(1, 3, 1, n),
            "x": x, "dx": dx, "domain": (a, b), "n": n, "bc": "periodic", "gamma": gamma}


def random_smooth_2d(nx=48, ny=40, seed=0, gamma=GAMMA, amp=0.2):
    """Smooth periodic 2D Euler data on [0,1]^2 (random low Fourier modes)."""
    rng = np.random.default_rng(seed)
    x, dx = cell_centres(0.0, 1.0, nx)
    y, dy = cell_centres(0.0, 1.0, ny)
    X, Y = np.meshgrid(x, y)
    def field(base):
        out = np.full_like(X, base)
        for kx in range(0, 3):
            for ky in range(0, 3):
                a, b = rng.normal(size=2) * amp / 3
                out += a * np.sin(2 * np.pi * (kx * X + ky * Y)) + b * np.cos(2 * np.pi * (kx * X + ky * Y))
        return out
    rho = field(1.0) + 0.5
    u = field(0.2)
    v = field(-0.1)
    p = field(1.0) + 0.5
    return {"system": "euler", "ndim": 2, "U": cons_2d(rho, u, v, p, gamma).reshape(1, 4, ny, nx),
            "dx": dx, "dy": dy, "nx": nx, "ny": ny, "bc": "periodic", "gamma": gamma}

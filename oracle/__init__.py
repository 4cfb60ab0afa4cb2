"""ctypes binding of the CPU oracle (test infrastructure only).

The oracle is the plain FP64 C++ restatement of WENO-ZA6 (arXiv 2603.26272,
Sections 2-4) that the CUDA library is checked against.  Only tests/, the
smoke check in __graft_entry__ and bench.py's CPU-baseline leg may import it.
It imports nothing from the CUDA package.
"""
import contextlib
import ctypes
import os

import numpy as np

from . import build as _build

_libs = {}
_variant = None


class OraGrid(ctypes.Structure):
    """Mirror of ora_grid in weno_oracle.h."""
    _fields_ = [
        ("system", ctypes.c_int32),
        ("ndim", ctypes.c_int32),
        ("nbatch", ctypes.c_int64),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("dy", ctypes.c_double),
        ("bc_x", ctypes.c_int32),
        ("bc_y", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("mu0", ctypes.c_double),
        ("p", ctypes.c_double),
        ("ai", ctypes.c_int32),
        ("alpha_mode", ctypes.c_int32),
        ("adv_speed", ctypes.c_double),
        ("order", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_G = ctypes.POINTER(OraGrid)


def lib():
    """The oracle library of the current rounding variant (built on demand)."""
    if _variant not in _libs:
        _libs[_variant] = _load(_build.build(variant=_variant))
    return _libs[_variant]


@contextlib.contextmanager
def rounding_variant(name):
    """Within the block every oracle call runs the build whose final sums
    (eq. (14), the projections on L, the back-projection on R) are taken in
    the opposite order ("reversed"): the same arithmetic, rounded
    differently.  None is the stock build."""
    global _variant
    assert name in _build.VARIANTS
    old = _variant
    _variant = name
    try:
        yield
    finally:
        _variant = old


def _load(path):
    L = ctypes.CDLL(path)
    L.ora_za6_flux.restype = ctypes.c_double
    L.ora_za6_flux.argtypes = [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_int, _D]
    L.ora_za6_flux_quad.restype = ctypes.c_double
    L.ora_za6_flux_quad.argtypes = [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int]
    L.ora_coefficients.restype = None
    L.ora_coefficients.argtypes = [_D]
    L.ora_za_flux.restype = ctypes.c_double
    L.ora_za_flux.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, ctypes.c_int]
    L.ora_coefficients_r.argtypes = [ctypes.c_int, _D]
    L.ora_operator_error.restype = ctypes.c_double
    L.ora_operator_error.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int]
    for name in ("ora_alpha",):
        getattr(L, name).argtypes = [_G, _D, _D]
    L.ora_roe_face.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D, _D]
    L.ora_rhs.argtypes = [_G, _D, _D, _D]
    L.ora_rhs_cell.argtypes = [_G, _D, _D, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _D]
    L.ora_cfl_dt.argtypes = [_G, _D, ctypes.c_double, _D]
    L.ora_ssprk3_step.argtypes = [_G, _D, _D]
    L.ora_solve.argtypes = [_G, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_int64, _D, _I64]
    L.ora_riemann_exact.argtypes = [ctypes.c_double] * 7 + [ctypes.c_double, ctypes.c_double,
                                                            ctypes.c_int64, _D, _D, _D, _D, _D]
    return L


def _p(a):
    return a.ctypes.data_as(_D)


class OracleError(RuntimeError):
    pass


def _check(code, what):
    if code == 0:
        return
    msg = {1: "bad argument", 2: "nonphysical state", 3: "max_steps reached"}.get(code, str(code))
    raise OracleError("%s: %s" % (what, msg))


def make_grid(system="euler", ndim=1, nbatch=1, nx=1, ny=1, dx=1.0, dy=1.0, bc_x="transmissive",
              bc_y="transmissive", gamma=1.4, eps=1e-40, mu0=1e-40, p=1.0, ai=1,
              alpha_mode="field", adv_speed=1.0, order=6):
    bcs = {"transmissive": 0, "periodic": 1}
    g = OraGrid()
    g.system = {"advection": 0, "euler": 1, "burgers": 2, "buckley_leverett": 3}[system]
    g.ndim = ndim
    g.nbatch = nbatch
    g.nx = nx
    g.ny = ny
    g.dx = dx
    g.dy = dy
    g.bc_x = bcs[bc_x]
    g.bc_y = bcs[bc_y]
    g.gamma = gamma
    g.eps = eps
    g.mu0 = mu0
    g.p = p
    g.ai = int(ai)
    g.alpha_mode = {"field": 0, "single": 1}[alpha_mode]
    g.adv_speed = adv_speed
    g.order = order
    return g


def ncomp(g):
    if g.system != 1:
        return 1
    return 3 if g.ndim == 1 else 4


def _state(g, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.size == g.nbatch * ncomp(g) * g.nx * g.ny, "state size mismatch"
    return U


def za6_flux(f, eps=1e-40, mu0=1e-40, p=1.0, ai=1, detail=False):
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (6,)
    if detail:
        d = np.zeros(16)
        lib().ora_za6_flux(_p(f), eps, mu0, p, int(ai), _p(d))
        return {"fk": d[0:4].copy(), "beta": d[4:9].copy(), "tau": d[9], "mu": d[10],
                "omega": d[11:15].copy(), "fhat": d[15]}
    return lib().ora_za6_flux(_p(f), eps, mu0, p, int(ai), None)


def za6_flux_quad(f, eps=1e-40, mu0=1e-40, p=1.0, ai=1):
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().ora_za6_flux_quad(_p(f), eps, mu0, p, int(ai))


def coefficients():
    out = np.zeros(64)
    lib().ora_coefficients(_p(out))
    return {"c6": out[0:6], "ck": out[6:18].reshape(4, 3), "d": out[18:22],
            "B0": out[22:31].reshape(3, 3), "B1": out[31:40].reshape(3, 3),
            "B2": out[40:49].reshape(3, 3), "Bd": out[49:58].reshape(3, 3), "ctau": out[58:64]}


def za_flux(order, f, eps=1e-40, mu0=1e-40, p=1.0, ai=1):
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (order,)
    return lib().ora_za_flux(int(order), _p(f), eps, mu0, p, int(ai))


def coefficients_r(order):
    r = order // 2
    n = 2 * r + (r + 1) * r + (r + 1) + (r + 1) * r * r + 2 * r
    out = np.zeros(n)
    _check(lib().ora_coefficients_r(int(order), _p(out)), "ora_coefficients_r")
    o = 0
    res = {}
    for name, size, shape in (("c2r", 2 * r, (2 * r,)), ("ck", (r + 1) * r, (r + 1, r)),
                              ("d", r + 1, (r + 1,)), ("B", (r + 1) * r * r, (r + 1, r, r)),
                              ("ctau", 2 * r, (2 * r,))):
        res[name] = out[o:o + size].reshape(shape)
        o += size
    return res


def operator_error(ncp, inv_dx, p=1.0, eps_variable=False, quad=False):
    return lib().ora_operator_error(int(ncp), int(inv_dx), float(p), int(eps_variable), int(quad))


def roe_face(UL, UR, dir=0, gamma=1.4):
    """Roe-averaged face state of two cells and its eigen-system (Section 4.2):
    dict with u, v, H, c, R (columns = right eigenvectors), L (= R^-1), lam."""
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    nc = UL.size
    assert UR.size == nc and nc in (3, 4)
    out = np.zeros(40)
    _check(lib().ora_roe_face(nc, int(dir), float(gamma), _p(UL), _p(UR), _p(out)),
           "ora_roe_face")
    return {"u": out[0], "v": out[1], "H": out[2], "c": out[3],
            "R": out[4:20].reshape(4, 4)[:nc, :nc].copy(),
            "L": out[20:36].reshape(4, 4)[:nc, :nc].copy(), "lam": out[36:36 + nc].copy()}


def alpha(g, U):
    U = _state(g, U)
    out = np.zeros(g.nbatch * 8)
    _check(lib().ora_alpha(ctypes.byref(g), _p(U), _p(out)), "ora_alpha")
    return out.reshape(g.nbatch, 2, 4)


def rhs(g, U, al=None):
    U = _state(g, U)
    if al is None:
        al = alpha(g, U)
    al = np.ascontiguousarray(al, dtype=np.float64)
    L = np.zeros_like(U)
    _check(lib().ora_rhs(ctypes.byref(g), _p(U), _p(al), _p(L)), "ora_rhs")
    return L


def rhs_cell(g, U, al, b, j, i):
    U = _state(g, U)
    al = np.ascontiguousarray(al, dtype=np.float64)
    out = np.zeros(ncomp(g))
    _check(lib().ora_rhs_cell(ctypes.byref(g), _p(U), _p(al), b, j, i, _p(out)), "ora_rhs_cell")
    return out


def cfl_dt(g, U, cfl):
    U = _state(g, U)
    dt = np.zeros(g.nbatch)
    _check(lib().ora_cfl_dt(ctypes.byref(g), _p(U), float(cfl), _p(dt)), "ora_cfl_dt")
    return dt


def ssprk3_step(g, U, dt):
    U = _state(g, U).copy()
    dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (g.nbatch,)))
    _check(lib().ora_ssprk3_step(ctypes.byref(g), _p(U), _p(dt)), "ora_ssprk3_step")
    return U


def solve(g, U, cfl, t_final, t0=0.0, max_steps=10**9, allow_max_steps=False):
    U = _state(g, U).copy()
    t = np.zeros(g.nbatch)
    steps = np.zeros(g.nbatch, dtype=np.int64)
    code = lib().ora_solve(ctypes.byref(g), _p(U), float(cfl), float(t0), float(t_final),
                           int(max_steps), _p(t), steps.ctypes.data_as(_I64))
    if not (code == 3 and allow_max_steps):
        _check(code, "ora_solve")
    return U, t, steps


def riemann_exact(left, right, x, t, x0=0.0, gamma=1.4):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.size
    rho, u, p, star = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(2)
    _check(lib().ora_riemann_exact(left[0], left[1], left[2], right[0], right[1], right[2],
                                   gamma, x0, t, n, _p(x), _p(rho), _p(u), _p(p), _p(star)),
           "ora_riemann_exact")
    return rho, u, p, star

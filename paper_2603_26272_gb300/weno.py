"""Thin ctypes binding of libweno (the C-ABI declared in include/weno.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libweno.so.  Device memory, streams and workspaces are PyTorch tensors
passed by pointer.  There is no CPU fallback: if the library is not built or
no GPU is present, the calls raise.
"""
import ctypes
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libweno.so")

WENO_OK, WENO_ERR_ARG, WENO_ERR_CUDA, WENO_ERR_NONPHYSICAL = 0, 1, 2, 3
WENO_ERR_NOMEM, WENO_ERR_TIMEOUT, WENO_ERR_MAXSTEPS = 4, 5, 6
STATUS_NAMES = {0: "WENO_OK", 1: "WENO_ERR_ARG", 2: "WENO_ERR_CUDA", 3: "WENO_ERR_NONPHYSICAL",
                4: "WENO_ERR_NOMEM", 5: "WENO_ERR_TIMEOUT", 6: "WENO_ERR_MAXSTEPS"}

SYSTEMS = {"advection": 0, "euler": 1, "burgers": 2, "buckley_leverett": 3}
BCS = {"transmissive": 0, "periodic": 1}
PRECISIONS = {"fp64": 0, "fp32_recon": 1}
ALPHA_MODES = {"field": 0, "single": 1}


class Desc(ctypes.Structure):
    """Mirror of weno_desc."""
    _fields_ = [
        ("system", ctypes.c_int32),
        ("ndim", ctypes.c_int32),
        ("nbatch", ctypes.c_int64),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("x0", ctypes.c_double),
        ("x1", ctypes.c_double),
        ("y0", ctypes.c_double),
        ("y1", ctypes.c_double),
        ("bc_x", ctypes.c_int32),
        ("bc_y", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("mu0", ctypes.c_double),
        ("p", ctypes.c_double),
        ("ai", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("alpha_mode", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("adv_speed", ctypes.c_double),
    ]

    @property
    def ncomp(self):
        return 1 if self.system != 1 else (3 if self.ndim == 1 else 4)

    @property
    def shape(self):
        return (self.nbatch, self.ncomp, self.ny, self.nx)


class WenoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


_lib = None
_VP = ctypes.c_void_p
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
_DESCP = ctypes.POINTER(Desc)


def lib():
    """Load libweno.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libweno.so is not built (run __graft_entry__.build() or "
                               "python paper_2603_26272_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        L.weno_workspace_bytes.restype = _SZ
        L.weno_workspace_bytes.argtypes = [_DESCP]
        L.weno_workspace_bytes_host.restype = _SZ
        L.weno_workspace_bytes_host.argtypes = [_DESCP]
        L.weno_wavespeeds.argtypes = [_DESCP, _VP, _VP, _VP, _VP, _SZ, _VP]
        L.weno_rhs.argtypes = [_DESCP, _VP, _VP, _VP, _SZ, _VP]
        L.weno_step.argtypes = [_DESCP, _VP, _D, _DP, _VP, _SZ, _VP]
        L.weno_solve.argtypes = [_DESCP, _VP, _D, _D, _I64, _DP, _I64P, _VP, _SZ, _VP]
        L.weno_solve_host.argtypes = [_DESCP, _VP, _D, _D, _I64, _DP, _I64P, _VP, _SZ, _VP]
        L.weno_sync_status.argtypes = [_DESCP, _VP, _SZ, _VP]
        L.weno_step_host.argtypes = [_DESCP, _VP, _D, _DP, _VP, _SZ, _VP]
        L.weno_last_error.restype = ctypes.c_char_p
        L.weno_last_error.argtypes = []
        L.weno_version.restype = ctypes.c_char_p
        L.weno_version.argtypes = []
        L.weno_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, _DP, _VP]
        L.weno_dd_begin.argtypes = [_DESCP, _I64, _VP, _VP, _VP, _VP, _SZ, _VP]
        L.weno_dd_speeds.argtypes = [_DESCP, _I64, ctypes.c_int, _VP, _SZ,
                                     ctypes.POINTER(ctypes.c_void_p)]
        L.weno_dd_stage.argtypes = [_DESCP, _I64, ctypes.c_int, _VP, _D, _VP, _VP, _VP, _VP, _VP,
                                    _SZ, _VP]
        for name in ("weno_dd_begin", "weno_dd_speeds", "weno_dd_stage"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("weno_wavespeeds", "weno_rhs", "weno_step", "weno_solve", "weno_solve_host",
                     "weno_sync_status", "weno_step_host", "weno_fma_rate"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(code):
    if code != WENO_OK:
        raise WenoError(code, lib().weno_last_error().decode())


def make_desc(system="euler", ndim=1, nbatch=1, nx=1, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
              bc_x="transmissive", bc_y="transmissive", gamma=1.4, cfl=0.5, eps=1e-40,
              mu0=1e-40, p=1.0, ai=True, precision="fp64", alpha_mode="field", adv_speed=1.0,
              order=6):
    d = Desc()
    d.system = SYSTEMS[system]
    d.ndim = ndim
    d.nbatch = nbatch
    d.nx = nx
    d.ny = ny
    d.x0, d.x1, d.y0, d.y1 = x0, x1, y0, y1
    d.bc_x = BCS[bc_x]
    d.bc_y = BCS[bc_y]
    d.gamma = gamma
    d.cfl = cfl
    d.eps = eps
    d.mu0 = mu0
    d.p = p
    d.ai = int(bool(ai))
    d.precision = PRECISIONS[precision]
    d.alpha_mode = ALPHA_MODES[alpha_mode]
    d.order = int(order)
    d.adv_speed = adv_speed
    return d


def workspace_bytes(desc, host=False):
    f = lib().weno_workspace_bytes_host if host else lib().weno_workspace_bytes
    n = f(ctypes.byref(desc))
    if n == 0:
        raise WenoError(WENO_ERR_ARG, lib().weno_last_error().decode())
    return n


def workspace(desc, device=None, host=False):
    """A device workspace tensor (uint8) big enough for desc."""
    n = workspace_bytes(desc, host)
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _state(desc, U):
    if not (isinstance(U, torch.Tensor) and U.is_cuda):
        raise TypeError("U must be a CUDA tensor")
    if U.dtype != torch.float64 or not U.is_contiguous():
        raise TypeError("U must be contiguous float64")
    if tuple(U.shape) != desc.shape:
        raise ValueError("U has shape %s, descriptor wants %s" % (tuple(U.shape), desc.shape))
    return ctypes.c_void_p(U.data_ptr())


def _ws(desc, ws, device, host=False):
    if ws is None:
        ws = workspace(desc, device, host)
    return ws, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())


def wavespeeds(desc, U, ws=None, stream=None):
    """(alpha [nbatch, 2, 4], dt [nbatch]) as device tensors (eq. (6), CFL rule)."""
    Up = _state(desc, U)
    ws, wp, wn = _ws(desc, ws, U.device)
    alpha = torch.empty((desc.nbatch, 2, 4), dtype=torch.float64, device=U.device)
    dt = torch.empty(desc.nbatch, dtype=torch.float64, device=U.device)
    _check(lib().weno_wavespeeds(ctypes.byref(desc), Up, ctypes.c_void_p(alpha.data_ptr()),
                                 ctypes.c_void_p(dt.data_ptr()), wp, wn, _stream(stream)))
    return alpha, dt


def rhs(desc, U, out=None, ws=None, stream=None):
    """L(U) of one Runge-Kutta stage (asynchronous)."""
    Up = _state(desc, U)
    if out is None:
        out = torch.empty_like(U)
    Op = _state(desc, out)
    ws, wp, wn = _ws(desc, ws, U.device)
    _check(lib().weno_rhs(ctypes.byref(desc), Up, Op, wp, wn, _stream(stream)))
    return out


def step(desc, U, dt=0.0, ws=None, stream=None, sync=True):
    """One SSP-RK3 step in place; returns the dt of each problem if sync."""
    Up = _state(desc, U)
    ws, wp, wn = _ws(desc, ws, U.device)
    if sync:
        used = (ctypes.c_double * desc.nbatch)()
        _check(lib().weno_step(ctypes.byref(desc), Up, float(dt), used, wp, wn, _stream(stream)))
        return list(used)
    _check(lib().weno_step(ctypes.byref(desc), Up, float(dt), None, wp, wn, _stream(stream)))
    return None


def solve(desc, U, t_final, t0=0.0, max_steps=2 ** 62, ws=None, stream=None,
          allow_max_steps=False):
    """Advance U in place from t0 to t_final; returns (t[nbatch], steps[nbatch]).
    With allow_max_steps, stopping at max_steps before t_final is not an
    error (continue with t0 = the returned t: the result is bitwise that of
    one call)."""
    Up = _state(desc, U)
    ws, wp, wn = _ws(desc, ws, U.device)
    t = (ctypes.c_double * desc.nbatch)()
    n = (ctypes.c_int64 * desc.nbatch)()
    code = lib().weno_solve(ctypes.byref(desc), Up, float(t0), float(t_final), int(max_steps),
                            t, n, wp, wn, _stream(stream))
    if not (allow_max_steps and code == WENO_ERR_MAXSTEPS):
        _check(code)
    return list(t), list(n)


def solve_host(desc, U_host, t_final, t0=0.0, max_steps=2 ** 62, ws=None, stream=None,
               device=None):
    """weno_solve_host on a CPU tensor (pinned for full copy bandwidth)."""
    if not isinstance(U_host, torch.Tensor) or U_host.is_cuda:
        raise TypeError("U_host must be a CPU tensor")
    if U_host.dtype != torch.float64 or not U_host.is_contiguous():
        raise TypeError("U_host must be contiguous float64")
    if tuple(U_host.shape) != desc.shape:
        raise ValueError("U_host has shape %s, descriptor wants %s" % (tuple(U_host.shape), desc.shape))
    ws, wp, wn = _ws(desc, ws, device or "cuda", host=True)
    t = (ctypes.c_double * desc.nbatch)()
    n = (ctypes.c_int64 * desc.nbatch)()
    _check(lib().weno_solve_host(ctypes.byref(desc), ctypes.c_void_p(U_host.data_ptr()),
                                 float(t0), float(t_final), int(max_steps), t, n, wp, wn,
                                 _stream(stream)))
    return list(t), list(n)


def step_host(desc, U_host, dt=0.0, ws=None, stream=None, device=None):
    """weno_step_host on a CPU tensor: copy in, one step, copy out; returns dt."""
    if not isinstance(U_host, torch.Tensor) or U_host.is_cuda:
        raise TypeError("U_host must be a CPU tensor")
    if U_host.dtype != torch.float64 or not U_host.is_contiguous():
        raise TypeError("U_host must be contiguous float64")
    if tuple(U_host.shape) != desc.shape:
        raise ValueError("U_host has shape %s, descriptor wants %s" % (tuple(U_host.shape), desc.shape))
    ws, wp, wn = _ws(desc, ws, device or "cuda", host=True)
    used = (ctypes.c_double * desc.nbatch)()
    _check(lib().weno_step_host(ctypes.byref(desc), ctypes.c_void_p(U_host.data_ptr()), float(dt),
                                used, wp, wn, _stream(stream)))
    return list(used)


def sync_status(desc, ws, stream=None):
    _check(lib().weno_sync_status(ctypes.byref(desc), ctypes.c_void_p(ws.data_ptr()),
                                  ctypes.c_size_t(ws.numel()), _stream(stream)))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def dd_begin(desc, nrows, U, send_lo, send_hi, ws, stream=None):
    """weno_dd_begin: local speed maxima of the strip U and its edge rows."""
    _check(lib().weno_dd_begin(ctypes.byref(desc), int(nrows), _ptr(U), _ptr(send_lo),
                               _ptr(send_hi), _ptr(ws), ctypes.c_size_t(ws.numel()),
                               _stream(stream)))


def dd_speeds(desc, nrows, stage, ws):
    """The strip's speed slot that `stage` reads, as an int64 view [nbatch, 8]
    of the workspace (bit patterns of non-negative doubles: integer max is
    the numeric max)."""
    out = ctypes.c_void_p(0)
    _check(lib().weno_dd_speeds(ctypes.byref(desc), int(nrows), int(stage), _ptr(ws),
                                ctypes.c_size_t(ws.numel()), ctypes.byref(out)))
    off = out.value - ws.data_ptr()
    n = desc.nbatch * 8 * 8
    return ws[off:off + n].view(torch.int64).view(desc.nbatch, 8)


def dd_stage(desc, nrows, stage, U, dt, halo_lo, halo_hi, send_lo, send_hi, ws, stream=None):
    """weno_dd_stage: Runge-Kutta stage `stage` of the strip U."""
    _check(lib().weno_dd_stage(ctypes.byref(desc), int(nrows), int(stage), _ptr(U), float(dt),
                               _ptr(halo_lo), _ptr(halo_hi), _ptr(send_lo), _ptr(send_hi),
                               _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream)))


FMA_KINDS = {"fp64": 0, "fp64_short_mantissa": 1, "fp32": 2}


def fma_rate(kind="fp64", iters=4096, stream=None):
    """Measured FMA throughput of the current GPU in FLOP/s (2 per FMA):
    'fp64' on full-mantissa operands, 'fp64_short_mantissa', or 'fp32'."""
    out = ctypes.c_double(0.0)
    _check(lib().weno_fma_rate(FMA_KINDS[kind], int(iters), ctypes.byref(out), _stream(stream)))
    return out.value


def version():
    return lib().weno_version().decode()


def desc_for(w, **kw):
    """Descriptor of a workload dict from paper_2603_26272_gb300.workloads."""
    U = w["U"]
    nb, _, ny, nx = U.shape
    dom = w.get("domain", (0.0, 1.0))
    if w["ndim"] == 1:
        args = dict(system=w["system"], ndim=1, nbatch=nb, nx=nx, ny=1, x0=dom[0], x1=dom[1],
                    bc_x=w["bc"], gamma=w.get("gamma", 1.4), cfl=w.get("cfl", 0.5))
    else:
        args = dict(system="euler", ndim=2, nbatch=nb, nx=nx, ny=ny, x0=dom[0], x1=dom[1],
                    y0=dom[0], y1=dom[1], bc_x=w["bc"], bc_y=w["bc"],
                    gamma=w.get("gamma", 1.4), cfl=w.get("cfl", 0.5))
    args.update(kw)
    return make_desc(**args)

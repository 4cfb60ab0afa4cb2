"""weno_rhs_noalloc: the right-hand side for callers that cannot allocate.

Some callers cannot call cudaMalloc or pass the library a workspace -- a
plug-in whose host application owns every device allocation, or a loop that
must never enter the allocator.  For them the library keeps a small fixed
scratch array of its own.  These tests call that entry point through the
C-ABI and check it against weno_rhs (which uses a caller workspace) on two
calls in a row with different data, within the stage tolerance the other GPU
tests use.  The file is collected last so that a failure here does not stop
a `-x` run before the other GPU tests have run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_26272_gb300 import weno
from paper_2603_26272_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STAGE_TOL = 1e-12


def _rel_err(a, b):
    nc = b.shape[1]
    scale_all = np.abs(b).max()
    worst = 0.0
    for k in range(nc):
        s = np.abs(b[:, k]).max()
        if s <= 1e-14 * scale_all:
            s = scale_all
        worst = max(worst, np.abs(a[:, k] - b[:, k]).max() / (s if s > 0 else 1.0))
    return worst


def _noalloc(d, U, out):
    f = weno.lib().weno_rhs_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(weno.Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return f(ctypes.byref(d), ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()),
             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    a = wl.quadrant_2d(n=70, seed=11)
    b = wl.quadrant_2d(n=70, seed=12)
    c = wl.quadrant_2d(n=70, seed=13)
    two_d = dict(a)
    two_d["U"] = np.ascontiguousarray(np.concatenate([a["U"], b["U"], c["U"]], axis=0)[:, :, :45, :])
    d2 = weno.desc_for(two_d, x1=70 * a["dx"], y1=45 * a["dy"])
    one_d = wl.riemann_batch(nbatch=5, n=400, seed=4)
    return [(d2, two_d["U"]), (weno.desc_for(one_d), one_d["U"])]


def test_noalloc_rhs_matches_workspace_rhs_on_two_calls():
    for d, U in _cases():  # two calls in a row, different shapes and data
        Ug = torch.from_numpy(U).cuda()
        ref = weno.rhs(d, Ug).cpu().numpy()
        out = torch.full_like(Ug, float("nan"))
        code = _noalloc(d, Ug, out)
        assert code == weno.WENO_OK, weno.lib().weno_last_error().decode()
        assert _rel_err(out.cpu().numpy(), ref) <= STAGE_TOL


def test_noalloc_rejects_a_batch_beyond_its_scratch():
    d = weno.make_desc(system="euler", ndim=1, nbatch=2000, nx=16)
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(d, U, out) == weno.WENO_ERR_ARG
    msg = weno.lib().weno_last_error().decode()
    assert "1020" in msg and "nbatch" in msg


def test_noalloc_reports_a_nonphysical_input_then_recovers():
    """A negative density is reported by this call (the entry point has no
    workspace to inspect later), with its problem and cell; the status word in
    the shared array is cleared again by the next call, which succeeds."""
    w = wl.riemann_batch(nbatch=3, n=200, seed=6)
    d = weno.desc_for(w)
    bad = w["U"].copy()
    bad[1, 0, 0, 77] = -0.5
    out = torch.empty(bad.shape, dtype=torch.float64, device="cuda")
    assert _noalloc(d, torch.from_numpy(bad).cuda(), out) == weno.WENO_ERR_NONPHYSICAL
    msg = weno.lib().weno_last_error().decode()
    assert "problem 1" in msg and "i=77" in msg, msg
    Ug = torch.from_numpy(w["U"]).cuda()
    ref = weno.rhs(d, Ug).cpu().numpy()
    assert _noalloc(d, Ug, out) == weno.WENO_OK, weno.lib().weno_last_error().decode()
    assert _rel_err(out.cpu().numpy(), ref) <= STAGE_TOL


def test_noalloc_takes_no_device_memory():
    """After a first call (which may load the kernels' code), further calls
    leave the device's free memory unchanged."""
    d, U = _cases()[0]
    Ug = torch.from_numpy(U).cuda()
    out = torch.empty_like(Ug)
    assert _noalloc(d, Ug, out) == weno.WENO_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _noalloc(d, Ug, out) == weno.WENO_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_at_the_batch_limit():
    """nbatch = 1020, where the status word and the speed slots fill the
    64 KiB array exactly."""
    w = wl.riemann_batch(nbatch=1020, n=24, seed=8)
    d = weno.desc_for(w)
    Ug = torch.from_numpy(np.ascontiguousarray(w["U"])).cuda()
    ref = weno.rhs(d, Ug).cpu().numpy()
    out = torch.full_like(Ug, float("nan"))
    assert _noalloc(d, Ug, out) == weno.WENO_OK, weno.lib().weno_last_error().decode()
    assert _rel_err(out.cpu().numpy(), ref) <= STAGE_TOL

"""The C-ABI library loads, exports every entry point of include/weno.h, and
its host-side argument checks work -- all without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2603_26272_gb300 import build as wbuild
from paper_2603_26272_gb300 import weno

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    wbuild.build()
    return weno.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "weno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(weno_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert {"weno_rhs", "weno_step", "weno_solve", "weno_workspace_bytes"} <= set(names)
    for n in names:
        assert hasattr(L, n), n


def test_descriptor_layout_matches_header():
    # the header's field order and types, as ctypes lays them out (C rules)
    assert ctypes.sizeof(weno.Desc) == 136
    assert weno.Desc.adv_speed.offset == 128
    src = open(os.path.join(ROOT, "include", "weno.h")).read()
    body = src[src.index("typedef struct weno_desc"):src.index("} weno_desc;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-z_0-9]+)\s*[;,]", body)
    assert names == [f[0] for f in weno.Desc._fields_]


def test_workspace_bytes_and_argument_checks(L):
    d = weno.make_desc(system="euler", ndim=2, nx=2048, ny=2048, bc_x="transmissive")
    n = weno.workspace_bytes(d)
    state = 8 * 4 * 2048 * 2048
    assert 2 * state <= n <= 2 * state + 16384
    assert weno.workspace_bytes(d, host=True) >= n + state
    bad = [dict(ndim=3), dict(nx=0), dict(ndim=1, ny=2), dict(gamma=1.0), dict(cfl=0.0),
           dict(eps=0.0), dict(precision="fp32_recon", ai=False), dict(system="advection", ndim=2, ny=4),
           dict(nbatch=70000), dict(x1=0.0), dict(order=5), dict(order=12), dict(order=2),
           dict(eps=1e-260), dict(mu0=1e-136), dict(eps=1e-250, mu0=1e-100),
           dict(eps=1e-200, mu0=1e-52),
           dict(order=8, precision="fp32_recon")]
    for kw in bad:
        args = dict(system="euler", ndim=2, nx=8, ny=8)
        args.update(kw)
        d = weno.make_desc(**args)
        assert L.weno_workspace_bytes(ctypes.byref(d)) == 0, kw
        assert L.weno_last_error().decode() != ""


def test_eps_mu0_lower_limits_are_accepted(L):
    for eps, mu0 in ((1e-250, 3e-26), (1e-40, 3e-131), (1e-40, 1e-40)):
        d = weno.make_desc(system="euler", ndim=2, nx=8, ny=8, eps=eps, mu0=mu0)
        assert L.weno_workspace_bytes(ctypes.byref(d)) > 0, (eps, mu0)


def test_every_order_of_the_family_is_accepted(L):
    for order in (0, 4, 6, 8, 10):
        d = weno.make_desc(system="euler", ndim=2, nx=8, ny=8, order=order)
        assert L.weno_workspace_bytes(ctypes.byref(d)) > 0, order


def test_entry_points_reject_bad_arguments_before_any_device_work(L):
    d = weno.make_desc(system="euler", ndim=1, nx=16)
    code = L.weno_rhs(ctypes.byref(d), None, None, None, 0, None)
    assert code == weno.WENO_ERR_ARG
    # a misaligned or too small workspace is refused
    code = L.weno_step(ctypes.byref(d), ctypes.c_void_p(256), 0.0, None, ctypes.c_void_p(4096), 8,
                       None)
    assert code == weno.WENO_ERR_NOMEM
    code = L.weno_step(ctypes.byref(d), ctypes.c_void_p(256), 0.0, None, ctypes.c_void_p(4100),
                       1 << 30, None)
    assert code == weno.WENO_ERR_ARG
    assert "aligned" in L.weno_last_error().decode()


def test_version(L):
    assert "sm_103a" in weno.version()


def test_binding_rejects_host_tensors_and_wrong_layouts():
    """The binding refuses a state that is not a contiguous float64 CUDA
    tensor of the descriptor's shape before it reaches the library (no CPU
    fallback: a host tensor is an error, not a slow path)."""
    import torch
    d = weno.make_desc(system="euler", ndim=1, nbatch=2, nx=16)
    assert d.shape == (2, 3, 1, 16)
    with pytest.raises(TypeError):
        weno.rhs(d, torch.zeros(d.shape, dtype=torch.float64))  # host memory
    with pytest.raises(TypeError):
        weno._state(d, torch.zeros(d.shape, dtype=torch.float32))
    with pytest.raises(TypeError):
        weno.step(d, torch.zeros(d.shape, dtype=torch.float64))

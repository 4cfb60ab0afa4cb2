"""GPU: the 2D solve split into strips of rows reproduces weno_step on the
whole grid bit for bit.

Each strip runs the stage kernel on its own rows with r ghost rows per side
from its neighbours (weno_dd_stage), and the GLF speeds of eq. (6) are the
maximum over all strips.  Every cell therefore gets the operands it gets in
the single-grid step.  Two ways of connecting the strips are covered: several
strips of one process stepped in lockstep (decomp.StripGroup: device copies,
no kernel waits for another) and two processes on this GPU exchanging their
rows through host memory over gloo (decomp.DistComm with host staging).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2603_26272_gb300 import decomp
from paper_2603_26272_gb300 import weno
from paper_2603_26272_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _problem(nx, ny, bc, seed=3, **kw):
    w = wl.quadrant_2d(n=max(nx, ny), seed=seed)
    U = np.ascontiguousarray(w["U"][:, :, :ny, :nx])
    d = weno.make_desc(system="euler", ndim=2, nx=nx, ny=ny, x0=0.0, x1=nx * w["dx"], y0=0.0,
                       y1=ny * w["dy"], bc_x=bc, bc_y=bc, **kw)
    return U, d


def _whole_grid(U, d, steps):
    V = torch.from_numpy(U).cuda()
    ws = weno.workspace(d)
    for _ in range(steps):
        weno.step(d, V, ws=ws, sync=False)
    weno.sync_status(d, ws)
    return V


@pytest.mark.parametrize("nstrips", [1, 2, 3])
@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_strip_group_is_bitwise_the_whole_grid(nstrips, bc):
    U, d = _problem(70, 53, bc)
    ref = _whole_grid(U, d, 10)
    grp = decomp.StripGroup(d, nstrips)
    parts = grp.split(torch.from_numpy(U).cuda())
    for _ in range(10):
        grp.step(parts)
    torch.cuda.synchronize()
    assert torch.equal(grp.join(parts), ref)


@pytest.mark.parametrize("kw", [dict(order=4), dict(order=10), dict(precision="fp32_recon"),
                                dict(alpha_mode="single"), dict(nbatch=2)])
def test_strip_group_other_schemes_and_batches(kw):
    kw = dict(kw)
    nb = kw.pop("nbatch", 1)
    U, d = _problem(48, 40, "transmissive", seed=5, **kw)
    if nb > 1:
        U2, _ = _problem(48, 40, "transmissive", seed=6)
        U = np.ascontiguousarray(np.concatenate([U, U2], axis=0))
        d.nbatch = nb
    ref = _whole_grid(U, d, 6)
    grp = decomp.StripGroup(d, 3)
    parts = grp.split(torch.from_numpy(U).cuda())
    for _ in range(6):
        grp.step(parts)
    torch.cuda.synchronize()
    assert torch.equal(grp.join(parts), ref)


def test_fixed_step_and_a_strip_of_r_rows():
    U, d = _problem(40, 9, "periodic")  # three strips of exactly 3 rows
    V = torch.from_numpy(U).cuda()
    ws = weno.workspace(d)
    weno.step(d, V, dt=1e-4, ws=ws)
    grp = decomp.StripGroup(d, 3)
    parts = grp.split(torch.from_numpy(U).cuda())
    grp.step(parts, dt=1e-4)
    torch.cuda.synchronize()
    assert torch.equal(grp.join(parts), V)


def test_strip_arguments_are_checked():
    U, d = _problem(40, 20, "transmissive")
    local = weno.Desc.from_buffer_copy(d)
    local.ny = 2
    ws = weno.workspace(local)
    V = torch.zeros((1, 4, 2, 40), dtype=torch.float64, device="cuda")
    with pytest.raises(weno.WenoError):  # fewer rows than the stencil's half-width
        weno.dd_begin(d, 2, V, None, None, ws)
    with pytest.raises(weno.WenoError):
        weno.dd_speeds(d, 20, 4, weno.workspace(d))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, bc, steps, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        U, d = _problem(64, 45, bc)
        j0, n = decomp.strip_rows(d.ny, world, 3)[rank]
        strip = decomp.Strip(d, j0, n)
        comm = decomp.DistComm(rank, world, strip.periodic, host_staging=True)
        V = torch.from_numpy(np.ascontiguousarray(U[:, :, j0:j0 + n, :])).cuda()
        for _ in range(steps):
            strip.step(V, comm)
        torch.cuda.synchronize()
        out[rank] = V.cpu().numpy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("bc", ["transmissive", "periodic"])
def test_two_processes_over_gloo_are_bitwise_the_whole_grid(bc):
    steps = 8
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, bc, steps, out), nprocs=2, join=True,
                           start_method="spawn")
        got = np.concatenate([out[0], out[1]], axis=2)
    U, d = _problem(64, 45, bc)
    ref = _whole_grid(U, d, steps).cpu().numpy()
    np.testing.assert_array_equal(got, ref)

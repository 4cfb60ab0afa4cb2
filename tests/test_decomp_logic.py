"""The domain decomposition's host logic on CPU, as gloo ranks.

A 2D Euler grid is split into strips of rows, one per rank (world sizes 2
and 3), and advanced three SSP-RK3 steps by paper_2603_26272_gb300.decomp:
the all-reduce of the GLF speed maxima (eq. (6) is a maximum over the whole
grid), the exchange of r = 3 rows with the neighbouring strips (periodic or
physical sides), and the stage sequencing.  The GPU kernels are stood in for
by the oracle applied to each strip extended by its halo rows (test
infrastructure; the product driver never imports it), so the gathered strips
must equal the oracle's own three steps on the whole grid bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(bc):
    from paper_2603_26272_gb300 import weno
    from paper_2603_26272_gb300 import workloads as wl
    w = wl.quadrant_2d(n=22, seed=3)
    U = np.ascontiguousarray(w["U"][:, :, :19, :])  # 22 x 19: uneven strips
    d = weno.make_desc(system="euler", ndim=2, nx=22, ny=19, x0=0.0, x1=22 * w["dx"], y0=0.0,
                       y1=19 * w["dy"], bc_x=bc, bc_y=bc)
    return U, d


class OracleOps:
    """The oracle in place of the strip kernels: the stage input extended by
    its halo rows (or by the transmissive ghost rows at a physical side), the
    oracle's L(U) with the global speeds, and the oracle's Runge-Kutta
    arithmetic (tests only)."""

    def __init__(self, desc):
        import oracle
        self.o = oracle
        self.d = desc
        self.dx = (desc.x1 - desc.x0) / desc.nx
        self.dy = (desc.y1 - desc.y0) / desc.ny
        self.bc = {0: "transmissive", 1: "periodic"}

    def grid(self, ny):
        return self.o.make_grid(ndim=2, nx=self.d.nx, ny=ny, dx=self.dx, dy=self.dy,
                                bc_x=self.bc[self.d.bc_x], bc_y="transmissive")

    def local_speeds(self, strip, U):
        return torch.from_numpy(self.o.alpha(self.grid(strip.nrows), U.numpy()).reshape(-1, 8).copy())

    def pack(self, strip, V):
        strip.send_lo.copy_(V[:, :, :strip.r])
        strip.send_hi.copy_(V[:, :, -strip.r:])

    def begin(self, strip, U):
        strip.Un = U.clone()
        strip.slots = [self.local_speeds(strip, U), None, None]
        self.pack(strip, U)

    def speeds(self, strip, stage):
        return strip.slots[stage - 1]

    def stage(self, strip, stage, U, dt, lo, hi):
        r = strip.r
        inp = {1: U, 2: getattr(strip, "U1", None), 3: getattr(strip, "U2", None)}[stage]
        lo = lo if lo is not None else inp[:, :, :1].repeat(1, 1, r, 1)
        hi = hi if hi is not None else inp[:, :, -1:].repeat(1, 1, r, 1)
        ext = torch.cat([lo, inp, hi], dim=2).numpy()
        al = strip.slots[stage - 1].numpy().reshape(-1, 2, 4)
        L = self.o.rhs(self.grid(strip.nrows + 2 * r), ext, al)[:, :, r:r + strip.nrows]
        if stage == 1:
            a = al[0]
            sx, sy = max(a[0, 0], a[0, 3]), max(a[1, 0], a[1, 3])
            strip.dt = dt if dt > 0 else self.d.cfl / (sx / self.dx + sy / self.dy)
        h = strip.dt
        Un = strip.Un.numpy()
        x = inp.numpy()
        if stage == 1:
            out = x + h * L
        elif stage == 2:
            out = 0.75 * Un + 0.25 * (strip.U1.numpy() + h * L)
        else:
            out = (1.0 / 3.0) * Un + (2.0 / 3.0) * (x + h * L)
        out = torch.from_numpy(np.ascontiguousarray(out))
        if stage == 1:
            strip.U1 = out
        elif stage == 2:
            strip.U2 = out
        else:
            U.copy_(out)
        if stage < 3:
            strip.slots[stage] = self.local_speeds(strip, out)
        self.pack(strip, out)


def _rank(rank, world, port, bc, steps, out):
    import torch.distributed as dist

    from paper_2603_26272_gb300 import decomp
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        U, d = _workload(bc)
        j0, n = decomp.strip_rows(d.ny, world, 3)[rank]
        strip = decomp.Strip(d, j0, n, device="cpu", ops=OracleOps(d))
        comm = decomp.DistComm(rank, world, strip.periodic)
        V = torch.from_numpy(np.ascontiguousarray(U[:, :, j0:j0 + n, :]))
        for _ in range(steps):
            strip.step(V, comm)
        out[rank] = V.numpy().copy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,bc", [(2, "transmissive"), (2, "periodic"), (3, "periodic"),
                                      (3, "transmissive")])
def test_strips_reproduce_the_whole_grid_bit_for_bit(world, bc):
    import oracle
    steps = 3
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, bc, steps, out), nprocs=world, join=True,
                           start_method="spawn")
        parts = [out[k] for k in range(world)]
    got = np.concatenate(parts, axis=2)
    U, d = _workload(bc)
    g = oracle.make_grid(ndim=2, nx=d.nx, ny=d.ny, dx=(d.x1 - d.x0) / d.nx,
                         dy=(d.y1 - d.y0) / d.ny, bc_x=bc, bc_y=bc)
    for _ in range(steps):
        U = oracle.ssprk3_step(g, U, oracle.cfl_dt(g, U, d.cfl))
    np.testing.assert_array_equal(got, U)


def test_strip_rows_and_neighbours():
    from paper_2603_26272_gb300 import decomp
    assert decomp.strip_rows(19, 2, 3) == [(0, 10), (10, 9)]
    assert decomp.strip_rows(9, 3, 3) == [(0, 3), (3, 3), (6, 3)]
    with pytest.raises(ValueError):
        decomp.strip_rows(8, 3, 3)
    assert decomp.neighbours(0, 3, False) == (None, 1)
    assert decomp.neighbours(2, 3, False) == (1, None)
    assert decomp.neighbours(0, 3, True) == (2, 1)
    assert decomp.neighbours(0, 1, True) == (0, 0)
    assert decomp.neighbours(0, 1, False) == (None, None)

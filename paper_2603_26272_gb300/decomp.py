"""Domain decomposition of a 2D Euler solve into strips of rows.

A grid of ny rows is cut into strips of consecutive rows, one per rank (GPU).
Each SSP-RK3 stage of the WENO-ZA6 right-hand side needs, beyond a strip's
own rows, r = 3 rows on each side (the 2r-point stencil of eq. (7) in y) and
the global Lax-Friedrichs speeds of eq. (6), a maximum over the WHOLE grid.
So per stage a strip

  1. replaces its local speed maxima (8 per problem) by their maximum over
     all strips (one all-reduce of 8 integers: the maxima are kept as the bit
     patterns of non-negative doubles, whose integer order is the numeric one),
  2. sends its first r rows to the strip below and its last r rows to the
     strip above, and receives theirs (a side of the global domain takes its
     boundary condition instead, unless it is periodic, where the last strip
     is the first one's neighbour),
  3. runs the stage kernel (weno_dd_stage), which writes the output's edge
     rows straight into the send buffers of the next exchange.

Every cell then sees the operands it sees in the single-grid solve, so the
strips reproduce weno_step bit for bit.  This module only moves buffers
between ranks and sequences the library calls; every step of the method runs
in libweno's kernels.

Communicators: `DistComm` over torch.distributed -- NCCL on device buffers,
or any backend with the buffers staged through host memory (gloo) --, and
`StripGroup`, which steps several strips of one process in lockstep (the
exchange is then a device copy, and no kernel ever waits for another).
"""
import numpy as np
import torch

from . import weno


def order_r(desc):
    return 3 if desc.order in (0, 6) else desc.order // 2


def strip_rows(ny, nstrips, r=3):
    """Rows (j0, nrows) of each strip: as even as possible, each >= r."""
    if nstrips < 1 or ny < nstrips * r:
        raise ValueError("%d rows cannot make %d strips of at least %d rows" % (ny, nstrips, r))
    base, extra = divmod(ny, nstrips)
    out, j0 = [], 0
    for k in range(nstrips):
        n = base + (1 if k < extra else 0)
        out.append((j0, n))
        j0 += n
    return out


def neighbours(rank, world, periodic):
    """(below, above): the ranks holding the rows under and over this strip,
    None at a non-periodic side of the global domain."""
    below = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return below, above


class LibOps:
    """The library calls of one strip (weno_dd_*)."""

    def begin(self, strip, U):
        weno.dd_begin(strip.desc, strip.nrows, U, strip.send_lo, strip.send_hi, strip.ws)

    def speeds(self, strip, stage):
        return weno.dd_speeds(strip.desc, strip.nrows, stage, strip.ws)

    def stage(self, strip, stage, U, dt, halo_lo, halo_hi):
        weno.dd_stage(strip.desc, strip.nrows, stage, U, dt, halo_lo, halo_hi, strip.send_lo,
                      strip.send_hi, strip.ws)


class Strip:
    """One strip of rows [j0, j0 + nrows) of the grid described by `desc`
    (the global descriptor), with its workspace and halo buffers."""

    def __init__(self, desc, j0, nrows, device="cuda", ops=None):
        self.desc = desc
        self.j0, self.nrows = int(j0), int(nrows)
        self.r = order_r(desc)
        self.ops = ops if ops is not None else LibOps()
        local = weno.Desc.from_buffer_copy(desc)
        local.ny = self.nrows
        self.local = local
        shape = (desc.nbatch, 4, self.r, desc.nx)
        self.ws = weno.workspace(local, device=device) if isinstance(self.ops, LibOps) else None
        mk = (lambda: torch.empty(shape, dtype=torch.float64, device=device))
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()

    @property
    def periodic(self):
        return self.desc.bc_y == weno.BCS["periodic"]

    def step(self, U, comm, dt=0.0):
        """One SSP-RK3 step of this strip, in place; `comm` connects it to
        the other strips (a DistComm)."""
        self.ops.begin(self, U)
        for s in (1, 2, 3):
            comm.max_(self.ops.speeds(self, s))
            lo, hi = comm.exchange(self)
            self.ops.stage(self, s, U, dt, lo, hi)


class DistComm:
    """torch.distributed between the ranks of one decomposed solve.  With
    host_staging the device buffers travel through host memory (a backend
    without device support, such as gloo)."""

    def __init__(self, rank, world, periodic, group=None, host_staging=False):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world, self.group = rank, world, group
        self.below, self.above = neighbours(rank, world, periodic)
        self.host = host_staging

    def max_(self, t):
        if self.world == 1:
            return
        if self.host:
            h = t.cpu()
            self.dist.all_reduce(h, op=self.dist.ReduceOp.MAX, group=self.group)
            t.copy_(h)
        else:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)

    def exchange(self, strip):
        """send_lo -> the strip below (its upper halo), send_hi -> the strip
        above (its lower halo); returns the halos (None at a physical side)."""
        lo = strip.recv_lo if self.below is not None else None
        hi = strip.recv_hi if self.above is not None else None
        if self.world == 1:  # periodic: this strip is its own neighbour
            if lo is not None:
                lo.copy_(strip.send_hi)
            if hi is not None:
                hi.copy_(strip.send_lo)
            return lo, hi
        d = self.dist
        if self.host:
            s_lo, s_hi = strip.send_lo.cpu(), strip.send_hi.cpu()
            r_lo = torch.empty_like(s_lo) if lo is not None else None
            r_hi = torch.empty_like(s_hi) if hi is not None else None
            reqs = []
            if self.above is not None:  # upward: tag 0
                reqs.append(d.isend(s_hi, self.above, group=self.group, tag=0))
            if self.below is not None:  # downward: tag 1
                reqs.append(d.isend(s_lo, self.below, group=self.group, tag=1))
            if lo is not None:
                reqs.append(d.irecv(r_lo, self.below, group=self.group, tag=0))
            if hi is not None:
                reqs.append(d.irecv(r_hi, self.above, group=self.group, tag=1))
            for q in reqs:
                q.wait()
            if lo is not None:
                lo.copy_(r_lo)
            if hi is not None:
                hi.copy_(r_hi)
            return lo, hi
        # device buffers (NCCL): sends and receives between one pair of ranks
        # match in the order they are posted, so post upward data first on
        # both sides (this also holds when below == above, two strips periodic)
        ops = []
        if self.above is not None:
            ops.append(d.P2POp(d.isend, strip.send_hi, self.above, group=self.group))
        if self.below is not None:
            ops.append(d.P2POp(d.isend, strip.send_lo, self.below, group=self.group))
        if lo is not None:
            ops.append(d.P2POp(d.irecv, lo, self.below, group=self.group))
        if hi is not None:
            ops.append(d.P2POp(d.irecv, hi, self.above, group=self.group))
        for q in d.batch_isend_irecv(ops):
            q.wait()
        return lo, hi


class StripGroup:
    """Several strips of one grid in one process, stepped in lockstep: the
    speed maxima meet by an element-wise maximum and the halos by device
    copies between the strips' buffers.  Each kernel runs to completion on
    its own; nothing waits for another launch."""

    def __init__(self, desc, nstrips, device="cuda"):
        self.desc = desc
        self.strips = [Strip(desc, j0, n, device) for j0, n in
                       strip_rows(desc.ny, nstrips, order_r(desc))]
        periodic = desc.bc_y == weno.BCS["periodic"]
        self.links = [neighbours(k, nstrips, periodic) for k in range(nstrips)]

    def split(self, U):
        """Views of the strips' rows of a global state [nbatch][4][ny][nx]
        (copied: each strip owns a contiguous buffer)."""
        return [U[:, :, s.j0:s.j0 + s.nrows, :].contiguous() for s in self.strips]

    def join(self, parts):
        return torch.cat(parts, dim=2)

    def step(self, parts, dt=0.0):
        for st, U in zip(self.strips, parts):
            st.ops.begin(st, U)
        for s in (1, 2, 3):
            sp = [st.ops.speeds(st, s) for st in self.strips]
            m = sp[0].clone()
            for t in sp[1:]:
                torch.maximum(m, t, out=m)
            for t in sp:
                t.copy_(m)
            halos = []
            for k, st in enumerate(self.strips):
                below, above = self.links[k]
                lo = hi = None
                if below is not None:
                    st.recv_lo.copy_(self.strips[below].send_hi)
                    lo = st.recv_lo
                if above is not None:
                    st.recv_hi.copy_(self.strips[above].send_lo)
                    hi = st.recv_hi
                halos.append((lo, hi))
            for st, U, (lo, hi) in zip(self.strips, parts, halos):
                st.ops.stage(st, s, U, dt, lo, hi)


def gather_rows(parts):
    """numpy concatenation of strips' states along y."""
    return np.concatenate([p.cpu().numpy() if hasattr(p, "cpu") else p for p in parts], axis=2)

"""Continuous-batching serving loop over the engine of libweno.

Requests are independent Euler solves (1D or 2D, FP64 or FP32
reconstruction, each to its own final time) arriving as a Poisson stream.
`serve_two_lane` is the serving loop: solves large enough to fill the GPU
alone run one at a time on a low-priority stream, and every other solve is
admitted to the continuous-batching engine (high-priority stream) as soon as
it arrives and the engine has room -- a free slot, work-list room and a free
block of its device arena (admission by free HBM) -- and advances there
with the other small solves.  `serve_continuous` puts every solve through
the engine (first come first served under a work budget).
`serve_one_at_a_time` is the baseline: the same requests, in arrival order,
each solved alone with weno_solve on the same GPU.

Argument marshalling and queueing only; every step of the method runs in the
CUDA kernels of libweno.so.
"""
import ctypes
import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import weno
from . import workloads as wl


class _EngineLib:
    def __init__(self):
        L = weno.lib()
        P = ctypes.POINTER
        L.weno_engine_control_bytes.restype = ctypes.c_size_t
        L.weno_engine_control_bytes.argtypes = [ctypes.c_int, ctypes.c_int64]
        L.weno_engine_slot_bytes.restype = ctypes.c_size_t
        L.weno_engine_slot_bytes.argtypes = [P(weno.Desc)]
        L.weno_engine_create.restype = ctypes.c_int
        L.weno_engine_create.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                         ctypes.c_int64, ctypes.c_void_p, P(ctypes.c_void_p)]
        L.weno_engine_admit.restype = ctypes.c_int
        L.weno_engine_admit.argtypes = [ctypes.c_void_p, P(weno.Desc), ctypes.c_void_p,
                                        ctypes.c_double, P(ctypes.c_int)]
        L.weno_engine_run.restype = ctypes.c_int
        L.weno_engine_run.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.weno_engine_set_priority.restype = ctypes.c_int
        L.weno_engine_set_priority.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.weno_engine_set_fast.restype = ctypes.c_int
        L.weno_engine_set_fast.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.weno_engine_poll.restype = ctypes.c_int
        L.weno_engine_poll.argtypes = [ctypes.c_void_p, P(ctypes.c_int), ctypes.c_int,
                                       P(ctypes.c_int), P(ctypes.c_int)]
        L.weno_engine_retire.restype = ctypes.c_int
        L.weno_engine_retire.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                         P(ctypes.c_double), P(ctypes.c_int64)]
        L.weno_engine_info.restype = ctypes.c_int
        L.weno_engine_info.argtypes = [ctypes.c_void_p, P(ctypes.c_size_t), P(ctypes.c_size_t),
                                       P(ctypes.c_int64)]
        L.weno_engine_destroy.restype = ctypes.c_int
        L.weno_engine_destroy.argtypes = [ctypes.c_void_p]
        self.L = L


_elib = None


def _lib():
    global _elib
    if _elib is None:
        _elib = _EngineLib()
    return _elib.L


FAST_STEPS = 4  # WENO_ENGINE_FAST_STEPS of include/weno.h


class Engine:
    """A serving engine over a device arena of `arena_bytes` (a torch tensor)."""

    def __init__(self, arena_bytes, max_slots=256, max_tiles=1 << 20, device="cuda"):
        L = _lib()
        ctl = L.weno_engine_control_bytes(max_slots, max_tiles)
        if arena_bytes < ctl + (1 << 20):
            raise ValueError("arena too small for the control region (%d bytes)" % ctl)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=device)
        self.max_slots = max_slots
        h = ctypes.c_void_p()
        weno._check(L.weno_engine_create(ctypes.c_void_p(self.arena.data_ptr()),
                                         ctypes.c_size_t(self.arena.numel()), max_slots,
                                         max_tiles, None, ctypes.byref(h)))
        self.h = h
        self.shapes = {}

    def slot_bytes(self, desc):
        return _lib().weno_engine_slot_bytes(ctypes.byref(desc))

    def admit(self, desc, U, t_final):
        """U: contiguous float64 numpy array in the layout of desc.  Returns
        the slot, or None when the engine is full (no slot, work-list room or
        arena block)."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        slot = ctypes.c_int(-1)
        code = _lib().weno_engine_admit(self.h, ctypes.byref(desc),
                                        U.ctypes.data_as(ctypes.c_void_p), float(t_final),
                                        ctypes.byref(slot))
        if code == weno.WENO_ERR_NOMEM:
            return None
        weno._check(code)
        self.shapes[slot.value] = U.shape
        return slot.value

    def run(self, nsteps):
        weno._check(_lib().weno_engine_run(self.h, int(nsteps)))

    def set_priority(self, priority):
        """CUDA stream priority of the engine's runs (lower = higher)."""
        weno._check(_lib().weno_engine_set_priority(self.h, int(priority)))

    def set_fast(self, slot, fast=True):
        """Fast slots take FAST_STEPS SSP-RK3 steps per engine step."""
        weno._check(_lib().weno_engine_set_fast(self.h, int(slot), int(bool(fast))))

    def poll(self):
        done = (ctypes.c_int * self.max_slots)()
        nd, na = ctypes.c_int(0), ctypes.c_int(0)
        weno._check(_lib().weno_engine_poll(self.h, done, self.max_slots, ctypes.byref(nd),
                                            ctypes.byref(na)))
        return [done[i] for i in range(min(nd.value, self.max_slots))], na.value

    def retire(self, slot, want_state=True):
        """Returns (U or None, t, steps, status code)."""
        U = np.empty(self.shapes[slot]) if want_state else None
        t, n = ctypes.c_double(0), ctypes.c_int64(0)
        code = _lib().weno_engine_retire(self.h, slot,
                                         U.ctypes.data_as(ctypes.c_void_p) if want_state else None,
                                         ctypes.byref(t), ctypes.byref(n))
        del self.shapes[slot]
        if code not in (weno.WENO_OK, weno.WENO_ERR_NONPHYSICAL):
            weno._check(code)
        return U, t.value, n.value, code

    def info(self):
        f, lg, nt = ctypes.c_size_t(0), ctypes.c_size_t(0), ctypes.c_int64(0)
        weno._check(_lib().weno_engine_info(self.h, ctypes.byref(f), ctypes.byref(lg),
                                            ctypes.byref(nt)))
        return {"heap_free": f.value, "heap_largest": lg.value, "tiles_in_use": nt.value}

    def close(self):
        if self.h:
            _lib().weno_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Request:
    rid: int
    arrival: float
    kind: str
    precision: str
    desc: weno.Desc
    U: np.ndarray
    t_final: float
    target_steps: int
    cells: int
    result: dict = field(default_factory=dict)


def make_requests(n, seed=5, rate=None, sides_2d=(128, 192, 256, 384, 512, 768, 1024),
                  n1d=(256, 16384), steps=(100, 1000), frac_2d=0.5, frac_fp32=0.5):
    """The serving workload: n independent solves, Poisson arrivals at `rate`
    per second (None: all at t = 0), half 1D Euler Riemann problems with N
    log-uniform in n1d, half 2D quadrant problems with a side from sides_2d;
    half FP64, half FP32 reconstruction; each with a final time reached in a
    target number of steps drawn uniformly from `steps`, converted with the
    problem's initial CFL step (computed on the GPU by weno_wavespeeds)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n) if rate else np.zeros(n)
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for k in range(n):
        is2d = rng.random() < frac_2d
        prec = "fp32_recon" if rng.random() < frac_fp32 else "fp64"
        target = int(rng.integers(steps[0], steps[1] + 1))
        sub = int(rng.integers(0, 2 ** 31))
        if is2d:
            side = int(sides_2d[rng.integers(0, len(sides_2d))])
            w = wl.quadrant_2d(n=side, seed=sub)
            cells = side * side
        else:
            nx = int(round(math.exp(rng.uniform(math.log(n1d[0]), math.log(n1d[1])))))
            w = wl.riemann_batch(nbatch=1, n=nx, seed=sub)
            cells = nx
        d = weno.desc_for(w, precision=prec)
        U = np.ascontiguousarray(w["U"])
        _, dt = weno.wavespeeds(d, torch.from_numpy(U).cuda())
        t_final = target * float(dt[0].item())
        reqs.append(Request(k, float(arrivals[k]), "2d" if is2d else "1d", prec, d, U, t_final,
                            target, cells))
    return reqs


# Relative cost of one cell-step by class (2D FP64 = 1), from the measured
# full-GPU rates of the stage kernels: 2D FP32-recon 2.9x faster; a 1D cell has
# one interface of three fields instead of two of four.
COST = {("2d", "fp64"): 1.0, ("2d", "fp32_recon"): 0.35, ("1d", "fp64"): 0.4,
        ("1d", "fp32_recon"): 0.15}


def work_units(r):
    return r.cells * COST.get((getattr(r, "kind", "2d"), getattr(r, "precision", "fp64")), 1.0)


def serve_continuous(engine, requests, steps_per_poll=2, keep_states=False, work_budget=None,
                     fast=None, fast_units=0.0, clock=time.perf_counter):
    """Continuous batching in real time.  Fills request.result with arrival,
    admit and completion times (seconds from the start), steps, status.

    Admission is first-come first-served under two limits: the engine must
    have room (slot, work list, arena block -- admission by free HBM; a
    request that does not fit lets later, smaller ones pass) and, when
    `work_budget` is set, the admitted solves' cost per step (work_units)
    must stay within it, so the GPU is kept full without stretching every
    solve by sharing it with all others.

    Every admitted solve advances one SSP-RK3 step per engine step, except
    the fast ones, which take FAST_STEPS (the engine repeats the launches over
    their tiles only).  `fast` chooses them: None (no fast slots), "light"
    (every solve costing at most `fast_units` per step), or "oldest" (the
    longest-admitted solves, in admission order, while their summed cost
    stays within `fast_units`) -- the second keeps the order of completion
    close to first-come first-served while the younger solves fill the GPU."""
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    waiting = []
    active = {}
    order = []  # admitted slots, oldest first
    marked = set()
    load = 0.0
    t0 = clock()

    def mark_fast():
        want = set()
        if fast == "light":
            want = {k for k in order if work_units(active[k]) <= fast_units}
        elif fast == "oldest":
            acc = 0.0
            for k in order:
                acc += work_units(active[k])
                if acc > fast_units:
                    break
                want.add(k)
        for k in marked - want:
            engine.set_fast(k, False)
        for k in want - marked:
            engine.set_fast(k, True)
        marked.clear()
        marked.update(want)

    while pending or waiting or active:
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        still = []
        changed = False
        for i, r in enumerate(waiting):
            wu = work_units(r)
            if work_budget is not None and active and load + wu > work_budget:
                still.extend(waiting[i:])  # keep arrival order behind the budget
                break
            slot = engine.admit(r.desc, r.U, r.t_final)
            if slot is None:
                still.append(r)
                continue
            r.result["admit"] = clock() - t0
            active[slot] = r
            order.append(slot)
            load += wu
            changed = True
        waiting = still
        if changed and fast:
            mark_fast()
        if active:
            engine.run(steps_per_poll)
            done, _ = engine.poll()
            for slot in done:
                U, t, n, code = engine.retire(slot, want_state=keep_states)
                r = active.pop(slot)
                order.remove(slot)
                marked.discard(slot)
                load -= work_units(r)
                r.result.update({"done": clock() - t0, "t": t, "steps": n, "status": code})
                if keep_states:
                    r.result["U"] = U
            if done and fast:
                mark_fast()
        elif pending:
            time.sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.01)))
    for r in requests:
        r.result["arrival"] = r.arrival
    return requests


def engine_tiles(r):
    """Work-list tiles of a request in the engine (16 x 15 cells in 2D, 127
    cells in 1D)."""
    d = r.desc
    if d.ndim == 2:
        return ((d.nx + 15) // 16) * ((d.ny + 14) // 15)
    return (d.nx + 126) // 127


def full_wave_tiles(device=None):
    """Tiles the GPU runs at once: 3 blocks of 16 x 15 cells per SM."""
    return 3 * torch.cuda.get_device_properties(device or torch.cuda.current_device()).multi_processor_count


class GpuLargeRunner:
    """Runs one large solve of the two-lane loop on the GPU: the state goes to
    the device, and weno_solve advances it in chunks of `chunk_steps` steps
    from the time reached (bitwise one call), each chunk on the stream of the
    oldest large solve or on the younger ones' stream, as `is_oldest()` says
    when the chunk starts.  One runner per worker thread."""

    def __init__(self, device, prio_oldest, prio_younger, chunk_steps=16, keep_states=False):
        torch.cuda.set_device(device)
        self.device = device
        self.s_old = torch.cuda.Stream(device=device, priority=prio_oldest)
        self.s_new = torch.cuda.Stream(device=device, priority=prio_younger)
        self.chunk = chunk_steps
        self.keep = keep_states

    def upload(self, r):
        with torch.cuda.stream(self.s_new):
            U = torch.from_numpy(r.U).to(self.device)
            ws = weno.workspace(r.desc, device=self.device)
        self.s_new.synchronize()
        return U, ws

    def run(self, r, state, is_oldest):
        """Returns (t reached, steps, status code, final state or None)."""
        U, ws = state
        t, steps, status = 0.0, 0, 0
        while t < r.t_final:
            st = self.s_old if is_oldest() else self.s_new
            try:
                tt, nn = weno.solve(r.desc, U, r.t_final, t0=t, max_steps=self.chunk, ws=ws,
                                    stream=st, allow_max_steps=True)
            except weno.WenoError as e:
                status = e.code
                break
            t, steps = tt[0], steps + nn[0]
            if nn[0] == 0:
                break
        return (t if status == 0 else float("nan")), steps, status, \
            (U.cpu().numpy() if self.keep else None)


def stream_priority_levels():
    """CUDA stream priorities of the two-lane loop (lower = higher): the
    engine when it goes first, the oldest large solve, the engine when it
    yields, the younger large solves."""
    least, greatest = torch.cuda.Stream.priority_range()

    def clamp(q):
        return min(max(q, greatest), least)

    return {"engine_first": greatest, "large_oldest": clamp(greatest + 1),
            "engine_yields": clamp(greatest + 2), "large_younger": least}


def serve_two_lane(engine, requests, large_tiles=None, large_workers=2, steps_per_poll=2,
                   keep_states=False, chunk_steps=16, bypass_s=0.0, priorities=None,
                   large_runner=None, clock=time.perf_counter):
    """Continuous batching with a lane for the solves that fill the GPU alone.

    A 2D solve of at least `large_tiles` tiles (default: one full wave of
    the GPU, so 384^2 and up) keeps every SM busy by itself: sharing the GPU
    with other such solves would only stretch each of them.  Those run one
    at a time, first come first served, through weno_solve on a stream of
    low priority, in worker threads: `large_workers` of them, so that a
    second large solve fills the SMs the first one's last wave of tiles and
    its host round trips leave idle (a 384^2 stage is 1.37 waves of the GPU
    in 16 x 15 tiles, 512^2 2.46).  The oldest large solve runs on a stream of higher priority
    than the younger ones (each solve goes in chunks of `chunk_steps` steps,
    weno_solve from the reached time, bitwise one call, and picks its stream
    per chunk), so it keeps the pace it has alone and first come first served
    holds for the large solves.  Every other solve (1D, small 2D) is
    admitted to the engine as soon as it arrives and there is room; the
    engine's stream has the highest priority, so its blocks take the places
    the large solve's blocks free and the small solves keep roughly the pace
    they have alone.  A small solve therefore never waits for a large one,
    and the GPU time a small solve alone would leave idle (a latency-bound
    stage on a few SMs) goes to the large solve.

    `bypass_s` bounds how far small solves may overtake a large one: while
    the engine's oldest solve arrived more than bypass_s after the oldest
    large solve in progress, the engine runs at a priority between the
    oldest large solve's and the younger ones' (the oldest large solve goes
    first, the engine fills what it leaves).  0 keeps arrival order between
    the lanes (every solve then finishes about as it would one at a time,
    or sooner); infinity lets small solves always go first.

    `priorities` (default stream_priority_levels()) and `large_runner` (a
    factory called once per worker thread; default: a GpuLargeRunner) are
    parameters so the host logic can run without a GPU.

    Fills request.result like serve_continuous (plus "lane")."""
    import queue
    import threading

    if large_tiles is None:
        large_tiles = full_wave_tiles()
    pr = priorities or stream_priority_levels()
    if large_runner is None:
        device = torch.cuda.current_device()

        def large_runner():
            return GpuLargeRunner(device, pr["large_oldest"], pr["large_younger"], chunk_steps,
                                  keep_states)
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    waiting = []
    active = {}
    big_q = queue.Queue()
    t0 = clock()
    errors = []
    order = []  # large solves in progress, oldest first
    arrival_of = {}
    lock = threading.Lock()
    engine.set_priority(pr["engine_first"])
    engine_prio = pr["engine_first"]

    def big_lane():
        runner = large_runner()
        while True:
            r = big_q.get()
            if r is None:
                return
            with lock:
                order.append(r.rid)
                arrival_of[r.rid] = r.arrival
            try:
                state = runner.upload(r)
                r.result["admit"] = clock() - t0

                def is_oldest(rid=r.rid):
                    with lock:
                        return order[0] == rid

                t, steps, status, U = runner.run(r, state, is_oldest)
                r.result.update({"t": t, "steps": steps, "status": status})
                if U is not None:
                    r.result["U"] = U
                r.result["done"] = clock() - t0
            except Exception as e:  # noqa: BLE001 -- reported by the main thread
                errors.append(e)
                r.result.update({"done": clock() - t0, "status": -1, "steps": 0})
            finally:
                with lock:
                    order.remove(r.rid)

    workers = [threading.Thread(target=big_lane, daemon=True) for _ in range(large_workers)]
    for wk in workers:
        wk.start()
    try:
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                r.result["lane"] = "large" if (r.desc.ndim == 2 and engine_tiles(r) >= large_tiles) \
                    else "engine"
                if r.result["lane"] == "large":
                    big_q.put(r)
                else:
                    waiting.append(r)
            still = []
            for r in waiting:
                slot = engine.admit(r.desc, r.U, r.t_final)
                if slot is None:
                    still.append(r)
                    continue
                r.result["admit"] = clock() - t0
                active[slot] = r
            waiting = still
            if waiting and not active:
                raise RuntimeError("request %d does not fit the empty engine (arena or work list "
                                   "too small)" % waiting[0].rid)
            if active:
                want = pr["engine_first"]
                with lock:
                    if order:
                        oldest_large = arrival_of[order[0]]
                        oldest_small = min(r.arrival for r in active.values())
                        if oldest_small > oldest_large + bypass_s:
                            want = pr["engine_yields"]
                if want != engine_prio:
                    engine.set_priority(want)
                    engine_prio = want
                engine.run(steps_per_poll)
                done, _ = engine.poll()
                for slot in done:
                    U, t, n, code = engine.retire(slot, want_state=keep_states)
                    r = active.pop(slot)
                    r.result.update({"done": clock() - t0, "t": t, "steps": n, "status": code})
                    if keep_states:
                        r.result["U"] = U
            elif pending:
                time.sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.005)))
    finally:
        for _ in workers:
            big_q.put(None)
        for wk in workers:
            wk.join()
        engine.set_priority(pr["engine_first"])
    if errors:
        raise errors[0]
    for r in requests:
        r.result["arrival"] = r.arrival
    return requests


def serve_one_at_a_time(requests, clock=time.perf_counter):
    """Baseline: each request solved alone (weno_solve), in arrival order."""
    t0 = clock()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        U = torch.from_numpy(r.U).cuda()
        r.result["admit"] = clock() - t0
        try:
            t, n = weno.solve(r.desc, U, r.t_final)
            r.result.update({"t": t[0], "steps": n[0], "status": 0})
        except weno.WenoError as e:
            r.result.update({"t": float("nan"), "steps": 0, "status": e.code})
        r.result["done"] = clock() - t0
        r.result["arrival"] = r.arrival
    return requests


def summarize(requests):
    lat = np.array([r.result["done"] - r.result["arrival"] for r in requests])
    span = max(r.result["done"] for r in requests) - min(r.result["arrival"] for r in requests)
    work = sum(r.cells * r.result["steps"] for r in requests)
    return {"requests": len(requests), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
            "makespan_s": float(span), "cell_updates": int(work),
            "throughput_cell_updates_per_s": float(work / span) if span > 0 else None,
            "failed": int(sum(1 for r in requests if r.result.get("status", 0) != 0))}

"""Host-side logic of the serving loop, with a fake engine (no GPU): arrival
order, admission by free memory with bypass, completion bookkeeping and the
latency summary."""
from dataclasses import dataclass, field

import numpy as np
import pytest

serve = pytest.importorskip("paper_2603_26272_gb300.serve")


@dataclass
class FakeReq:
    rid: int
    arrival: float
    size: int
    steps_needed: int
    cells: int = 100
    desc: object = None
    U: object = None
    t_final: float = 1.0
    result: dict = field(default_factory=dict)


class FakeEngine:
    """Capacity in 'bytes'; each run() step advances every admitted request."""

    def __init__(self, capacity):
        self.capacity = capacity
        self.used = 0
        self.slots = {}
        self.next = 0
        self.admitted = []
        self.fast_log = []

    def admit(self, desc, U, t_final):
        r = desc
        if self.used + r.size > self.capacity:
            return None
        self.used += r.size
        s = self.next
        self.next += 1
        self.slots[s] = [r, 0]
        self.admitted.append(r.rid)
        return s

    fast = ()

    def set_fast(self, slot, fast=True):
        self.fast = tuple(sorted(set(self.fast) - {slot} | ({slot} if fast else set())))
        self.fast_log.append((slot, fast))

    def run(self, n):
        for s, v in self.slots.items():
            v[1] += n * (serve.FAST_STEPS if s in self.fast else 1)

    def poll(self):
        return [s for s, v in self.slots.items() if v[1] >= v[0].steps_needed], len(self.slots)

    def retire(self, slot, want_state=True):
        self.fast = tuple(x for x in self.fast if x != slot)
        r, n = self.slots.pop(slot)
        self.used -= r.size
        return None, 1.0, r.steps_needed, 0


def _reqs():
    rs = [FakeReq(0, 0.0, 6, 10), FakeReq(1, 0.0, 6, 4), FakeReq(2, 0.0, 3, 4),
          FakeReq(3, 0.001, 2, 2), FakeReq(4, 0.002, 9, 3)]
    for r in rs:
        r.desc = r
    return rs


def test_admission_order_and_bypass():
    eng = FakeEngine(capacity=10)
    rs = _reqs()
    serve.serve_continuous(eng, rs, steps_per_poll=1)
    # request 1 (size 6) does not fit beside request 0; request 2 (size 3) passes it
    assert eng.admitted.index(2) < eng.admitted.index(1)
    assert sorted(eng.admitted) == [0, 1, 2, 3, 4]
    for r in rs:
        assert r.result["done"] >= r.result["admit"] >= r.result["arrival"] - 1e-9
        assert r.result["status"] == 0


def test_summary_percentiles():
    rs = _reqs()
    for k, r in enumerate(rs):
        r.result = {"arrival": r.arrival, "done": r.arrival + 0.1 * (k + 1), "steps": 5, "status": 0}
    s = serve.summarize(rs)
    lat = [0.1, 0.2, 0.3, 0.4, 0.5]
    assert s["p50_latency_s"] == pytest.approx(np.percentile(lat, 50))
    assert s["p99_latency_s"] == pytest.approx(np.percentile(lat, 99))
    assert s["cell_updates"] == 5 * 100 * 5
    assert s["failed"] == 0


def test_fast_oldest_marks_the_longest_admitted_within_the_cost_cap():
    # cost per step = cells (2D FP64 weight 1): caps 250 -> the two oldest
    rs = [FakeReq(k, 0.0, 1, 40 - 5 * k, cells=100) for k in range(5)]
    for r in rs:
        r.desc = r
    eng = FakeEngine(capacity=100)
    serve.serve_continuous(eng, rs, steps_per_poll=1, fast="oldest", fast_units=250.0)
    first = [s for s, f in eng.fast_log if f][:2]
    assert first == [0, 1]  # slots of requests 0 and 1 (admitted first)
    assert all(r.result["status"] == 0 for r in rs)
    # request 0 needs 40 steps; as a fast slot it finishes in 10 engine steps,
    # before request 4 (20 steps, normal while the two oldest are present)
    assert rs[0].result["done"] <= rs[4].result["done"]


def test_fast_light_marks_cheap_requests_only():
    rs = [FakeReq(0, 0.0, 1, 8, cells=1000), FakeReq(1, 0.0, 1, 8, cells=10),
          FakeReq(2, 0.0, 1, 8, cells=20)]
    for r in rs:
        r.desc = r
    eng = FakeEngine(capacity=100)
    serve.serve_continuous(eng, rs, steps_per_poll=1, fast="light", fast_units=50.0)
    assert sorted(s for s, f in eng.fast_log if f) == [1, 2]


def test_engine_tile_count_matches_the_library_constants():
    """serve.engine_tiles decides which solves fill the GPU alone from the
    engine's tile shape; the shape is a constant of the CUDA library
    (kEngineTX, kEngineTY, kEngine1DCells in csrc/weno_internal.h), so the
    two must agree."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(serve.__file__), "csrc", "weno_internal.h")).read()
    tx = int(re.search(r"kEngineTX\s*=\s*(\d+)", src).group(1))
    ty = int(re.search(r"kEngineTY\s*=\s*(\d+)", src).group(1))
    threads = int(re.search(r"kEngineThreads\s*=\s*(\d+)", src).group(1))
    cells1d = threads - 1 if re.search(r"kEngine1DCells\s*=\s*kEngineThreads\s*-\s*1", src) \
        else int(re.search(r"kEngine1DCells\s*=\s*(\d+)", src).group(1))

    @dataclass
    class D:
        ndim: int
        nx: int
        ny: int

    @dataclass
    class R:
        desc: object

    for nx, ny in [(128, 128), (384, 384), (1024, 1024), (100, 37)]:
        assert serve.engine_tiles(R(D(2, nx, ny))) == -(-nx // tx) * -(-ny // ty)
    for n in (256, 1600, 16384):
        assert serve.engine_tiles(R(D(1, n, 1))) == -(-n // cells1d)

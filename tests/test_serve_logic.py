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

    def run(self, n):
        for v in self.slots.values():
            v[1] += n

    def poll(self):
        return [s for s, v in self.slots.items() if v[1] >= v[0].steps_needed], len(self.slots)

    def retire(self, slot, want_state=True):
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

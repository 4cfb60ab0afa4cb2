"""Host logic of the two-lane serving loop on CPU (no GPU): a fake engine for
the small solves and a fake runner for the large ones.  Checks the lane
split by tile count, first come first served in the large lane, which large
solve is the oldest while two run at once, the engine's priority with and
without the bypass bound, and that every request completes with its lane."""
import threading
import time
from dataclasses import dataclass, field

import pytest

serve = pytest.importorskip("paper_2603_26272_gb300.serve")

PRIO = {"engine_first": -5, "large_oldest": -4, "engine_yields": -3, "large_younger": 0}


@dataclass
class FakeDesc:
    ndim: int
    nx: int
    ny: int


@dataclass
class FakeReq:
    rid: int
    arrival: float
    desc: FakeDesc
    work: int  # engine steps (small) or runner chunks (large)
    U: object = None
    t_final: float = 1.0
    result: dict = field(default_factory=dict)


class FakeEngine:
    def __init__(self):
        self.slots = {}
        self.next = 0
        self.priorities = []

    def set_priority(self, p):
        self.priorities.append(p)

    def admit(self, desc, U, t_final):
        s = self.next
        self.next += 1
        self.slots[s] = [desc.req, 0]
        return s

    def run(self, n):
        time.sleep(0.002)
        for v in self.slots.values():
            v[1] += n

    def poll(self):
        return [s for s, v in self.slots.items() if v[1] >= v[0].work], len(self.slots)

    def retire(self, slot, want_state=True):
        r, n = self.slots.pop(slot)
        return None, r.t_final, n, 0


class FakeRunner:
    """Each chunk sleeps 10 ms and records whether its solve was the oldest."""
    lock = threading.Lock()
    log = []

    def upload(self, r):
        with FakeRunner.lock:
            FakeRunner.log.append(("start", r.rid, time.perf_counter()))
        return None

    def run(self, r, state, is_oldest):
        for _ in range(r.work):
            with FakeRunner.lock:
                FakeRunner.log.append(("chunk", r.rid, is_oldest()))
            time.sleep(0.01)
        return r.t_final, 16 * r.work, 0, None


def _requests():
    # large: 2D 400 x 400 (625 tiles of 16 x 16); small: 2D 64^2 and 1D
    spec = [(0.00, "L", 6), (0.01, "S", 30), (0.02, "L", 3), (0.03, "S1", 20), (0.05, "L", 2),
            (0.08, "S", 10), (0.10, "S1", 15)]
    out = []
    for k, (t, kind, w) in enumerate(spec):
        d = FakeDesc(2, 400, 400) if kind == "L" else (FakeDesc(2, 64, 64) if kind == "S"
                                                        else FakeDesc(1, 3000, 1))
        r = FakeReq(k, t, d, w)
        d.req = r
        out.append(r)
    return out


def _serve(workers, bypass):
    FakeRunner.log = []
    eng = FakeEngine()
    reqs = _requests()
    serve.serve_two_lane(eng, reqs, large_tiles=456, large_workers=workers, bypass_s=bypass,
                         priorities=PRIO, large_runner=FakeRunner)
    return eng, reqs


def test_lanes_and_completion():
    eng, reqs = _serve(2, 0.0)
    for r in reqs:
        assert r.result["lane"] == ("large" if r.desc.nx == 400 else "engine"), r.rid
        assert r.result["status"] == 0
        assert r.result["done"] >= r.result["admit"] >= r.arrival - 1e-3
    assert eng.priorities[0] == PRIO["engine_first"] and eng.priorities[-1] == PRIO["engine_first"]


def test_large_lane_is_first_come_first_served():
    _serve(1, 0.0)
    starts = [rid for kind, rid, _ in FakeRunner.log if kind == "start"]
    assert starts == [0, 2, 4]
    # one worker: every chunk belongs to the oldest large solve
    assert all(old for kind, _, old in FakeRunner.log if kind == "chunk")


def test_two_workers_mark_only_the_oldest():
    _serve(2, 0.0)
    chunks = [(rid, old) for kind, rid, old in FakeRunner.log if kind == "chunk"]
    # solve 2 starts while 0 runs and is not the oldest until 0 is done
    done0 = max(i for i, (rid, _) in enumerate(chunks) if rid == 0)
    assert any(rid == 2 and not old for rid, old in chunks[:done0])
    assert all(old for rid, old in chunks if rid == 0)


def test_engine_yields_only_with_the_bypass_bound():
    eng, _ = _serve(2, 0.0)
    assert PRIO["engine_yields"] in eng.priorities  # small solves arrived after a large one
    eng, _ = _serve(2, float("inf"))
    assert set(eng.priorities) == {PRIO["engine_first"]}

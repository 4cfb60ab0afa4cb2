"""The serving engine: continuous batching of independent solves.

Every admitted problem advances with its own CFL step to its own final time,
on the same kernels as a solve alone, so its result must be bitwise the one
it gets alone (same steps, same final time, same state) whatever else shares
the GPU -- including a poisoned neighbour that fails.  Admission is by free
arena memory.
"""
import numpy as np
import pytest
import torch

from paper_2603_26272_gb300 import serve
from paper_2603_26272_gb300 import weno
from paper_2603_26272_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _alone(r):
    U = torch.from_numpy(r.U).cuda()
    t, n = weno.solve(r.desc, U, r.t_final)
    return U.cpu().numpy(), t[0], n[0]


def test_alone_equals_in_the_mix():
    reqs = serve.make_requests(10, seed=21, sides_2d=(40, 64, 100), n1d=(60, 3000), steps=(15, 60))
    eng = serve.Engine(arena_bytes=512 << 20, max_slots=32)
    serve.serve_continuous(eng, reqs, steps_per_poll=3, keep_states=True)
    kinds = set()
    for r in reqs:
        U, t, n = _alone(r)
        assert r.result["status"] == 0
        assert r.result["steps"] == n and r.result["t"] == t
        assert np.array_equal(r.result["U"], U), r.rid
        kinds.add((r.kind, r.precision))
    assert len(kinds) >= 3
    eng.close()


@pytest.mark.parametrize("bypass", [float("inf"), 0.0])
def test_two_lane_results_equal_alone(bypass):
    """The serving loop's two lanes: solves that fill a full wave of tiles run
    one at a time on a low-priority stream (here: the 2D side-400 requests,
    large_tiles lowered to 600), the others through the high-priority
    engine -- or, with bypass 0, below the oldest large solve, the engine's
    runs switching streams; every result is bitwise the solve alone, and
    both lanes are used while requests arrive over time."""
    reqs = serve.make_requests(12, seed=25, rate=40.0, sides_2d=(40, 64, 400), n1d=(60, 3000),
                               steps=(15, 40))
    eng = serve.Engine(arena_bytes=512 << 20, max_slots=32)
    serve.serve_two_lane(eng, reqs, large_tiles=600, keep_states=True, bypass_s=bypass)
    lanes = set()
    for r in reqs:
        U, t, n = _alone(r)
        assert r.result["status"] == 0
        assert r.result["steps"] == n and r.result["t"] == t
        assert np.array_equal(r.result["U"], U), r.rid
        assert r.result["done"] >= r.result["admit"] >= r.arrival - 1e-3
        lanes.add(r.result["lane"])
    assert lanes == {"large", "engine"}
    eng.close()


@pytest.mark.parametrize("fast,units", [("light", 3000.0), ("oldest", 8000.0)])
def test_fast_slots_equal_alone(fast, units):
    """Fast slots take several SSP-RK3 steps per engine step (the engine
    repeats the launches over their tiles); the results stay bitwise those of
    the solve alone, for the fast and the normal slots."""
    reqs = serve.make_requests(10, seed=24, sides_2d=(40, 64, 100), n1d=(60, 3000), steps=(15, 60))
    eng = serve.Engine(arena_bytes=512 << 20, max_slots=32)
    serve.serve_continuous(eng, reqs, steps_per_poll=2, keep_states=True, fast=fast,
                           fast_units=units)
    for r in reqs:
        U, t, n = _alone(r)
        assert r.result["status"] == 0
        assert r.result["steps"] == n and r.result["t"] == t
        assert np.array_equal(r.result["U"], U), r.rid
    eng.close()


def test_fast_slot_advances_several_steps_per_engine_step():
    w = wl.riemann_batch(nbatch=1, n=500, seed=3)
    d = weno.desc_for(w)
    eng = serve.Engine(arena_bytes=64 << 20, max_slots=4, max_tiles=4096)
    a = eng.admit(d, w["U"], 1e9)
    b = eng.admit(d, w["U"], 1e9)
    eng.set_fast(b)
    eng.run(3)
    eng.poll()
    _, _, na, _ = eng.retire(a, want_state=False)
    _, _, nb, _ = eng.retire(b, want_state=False)
    assert na == 3 and nb == 3 * serve.FAST_STEPS
    eng.close()


def test_poisoned_request_fails_alone():
    reqs = serve.make_requests(6, seed=22, sides_2d=(48,), n1d=(100, 400), steps=(20, 40))
    bad = reqs[2]
    bad.U = bad.U.copy()
    bad.U.reshape(-1)[bad.U.size // 7] = -1.0  # negative density somewhere
    eng = serve.Engine(arena_bytes=256 << 20, max_slots=16)
    serve.serve_continuous(eng, reqs, steps_per_poll=2, keep_states=True)
    assert bad.result["status"] == weno.WENO_ERR_NONPHYSICAL
    for r in reqs:
        if r is bad:
            continue
        U, t, n = _alone(r)
        assert r.result["status"] == 0 and r.result["steps"] == n
        assert np.array_equal(r.result["U"], U)
    eng.close()


def test_admission_by_free_arena_memory():
    w = wl.quadrant_2d(n=128, seed=3)
    d = weno.desc_for(w)
    probe = serve.Engine(arena_bytes=64 << 20, max_slots=4, max_tiles=4096)
    per = probe.slot_bytes(d)
    ctl = serve._lib().weno_engine_control_bytes(4, 4096)
    probe.close()
    eng = serve.Engine(arena_bytes=ctl + 2 * per + 4096, max_slots=4, max_tiles=4096)
    s0 = eng.admit(d, w["U"], 1e-3)
    s1 = eng.admit(d, w["U"], 1e-3)
    assert s0 is not None and s1 is not None
    assert eng.admit(d, w["U"], 1e-3) is None  # no arena left
    assert eng.info()["heap_largest"] < per
    eng.retire(s0, want_state=False)
    s2 = eng.admit(d, w["U"], 1e-3)
    assert s2 is not None
    eng.run(50)
    done, active = eng.poll()
    assert active == 2 and sorted(done) == sorted([s1, s2])
    for s in done:
        _, t, n, code = eng.retire(s, want_state=False)
        assert code == 0 and t == 1e-3
    assert eng.info()["tiles_in_use"] == 0
    eng.close()


def test_poisson_stream_completes_and_matches():
    reqs = serve.make_requests(16, seed=23, rate=400.0, sides_2d=(32, 64), n1d=(64, 1024),
                               steps=(10, 40))
    eng = serve.Engine(arena_bytes=256 << 20, max_slots=8)
    serve.serve_continuous(eng, reqs, steps_per_poll=2, keep_states=True)
    s = serve.summarize(reqs)
    assert s["failed"] == 0 and s["p99_latency_s"] >= s["p50_latency_s"] > 0
    for r in reqs[::5]:
        U, t, n = _alone(r)
        assert np.array_equal(r.result["U"], U)
    eng.close()

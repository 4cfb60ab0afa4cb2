"""The benchmark's multi-rank logic on CPU: two gloo ranks, as under
torchrun --nproc-per-node 2.  Each rank advances its own replica (no
collective on the data path); the whole-job number takes the slowest rank's
timed region and every rank's cell-updates, and only rank 0 prints.  The
reference arm does no work on ranks other than 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        elapsed = 100.0 + 50.0 * rank  # rank 1 is the slower one
        t_max, value = bench.job_timing(elapsed, world, cells=1000, steps=10, dist=dist)
        out[rank] = (t_max, value)
    finally:
        dist.destroy_process_group()


def test_job_timing_takes_the_slowest_rank_and_all_ranks_work():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        t_max, value = res[rank]
        assert t_max == 150.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.150)


def test_single_rank_timing():
    import bench
    t_max, value = bench.job_timing(40.0, 1, cells=4, steps=5)
    assert t_max == 40.0 and value == pytest.approx(4 * 5 / 0.04)


def test_reference_arm_is_silent_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_prints_one_line_on_rank_0():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0

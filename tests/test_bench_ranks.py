"""The N > 1 path of bench.py on CPU: every rank advances its own replica, the
job time is the maximum over ranks (gloo, world size 2) and only rank 0 of the
reference arm prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 10.0 + 5.0 * rank          # rank 1 is the slow one
        job = bench.job_time_ms(local, world, dist, device="cpu")
        q.put((rank, job, bench.job_value(1000, 4, world, job)))
    finally:
        dist.destroy_process_group()


def test_job_time_is_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, job, value in res:
        assert job == 15.0
        # 2 replicas x 1000 nodes x 4 steps in 15 ms
        assert value == pytest.approx(2 * 1000 * 4 / 15e-3, rel=1e-15)


def test_single_rank_needs_no_process_group():
    assert bench.job_time_ms(3.5, 1) == 3.5
    assert bench.job_value(10, 2, 1, 1.0) == pytest.approx(2e4)


def _reference(env_rank, world):
    env = dict(os.environ, RANK=str(env_rank), WORLD_SIZE=str(world), LOCAL_RANK=str(env_rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)


def test_reference_arm_prints_on_rank_zero_only():
    r1 = _reference(1, 2)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference(0, 2)
    assert r0.returncode == 0
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0

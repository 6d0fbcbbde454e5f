"""The multi-rank path of bench.py on the CPU: two gloo ranks time different
amounts, the whole-job rate uses the slowest rank's time and counts both ranks'
units, and under torchrun the reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    value, ms = bench.whole_job_rate(10.0 * (rank + 1), 100, 5, world)
    out.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in got:
        assert ms == pytest.approx(20.0)
        assert value == pytest.approx(100 * 2 * 5 / 0.020)


def test_reference_arm_prints_from_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.whole_job_rate(40.0, 1000, 4, 1)
    assert ms == 40.0 and value == pytest.approx(1000 * 4 / 0.040)

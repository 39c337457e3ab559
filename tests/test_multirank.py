"""CPU tests of the benchmark's multi-rank path: two gloo ranks on 127.0.0.1
reduce the per-rank timings (maximum) and marker counts (sum) the way the
benchmark's JSON line needs them, and the reference arm leaves every rank but
rank 0 without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.rank_reduce(1.5 + rank, world, dist.ReduceOp.MAX, "cpu")
    n = bench.rank_reduce(1000 * (rank + 1), world, dist.ReduceOp.SUM, "cpu")
    q.put((rank, ms, n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_times_and_counts():
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [2.5, 2.5]          # slowest rank's time
    assert [g[2] for g in got] == [3000.0, 3000.0]    # all ranks' markers


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""

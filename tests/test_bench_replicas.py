"""Replicas path of bench.py on CPU: two gloo ranks, each with its own time; the
job is timed by the slowest replica and the rate sums the replicas' units."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
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
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = bench.replica_max(dist, 10.0 + 3.0 * rank, "cpu")
    v = bench.whole_job_rate(world, 1000, 5, m * 1e-3)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == 13.0
        assert v == pytest.approx(2 * 1000 * 5 / 13.0e-3 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(None, 7.5, "cpu") == 7.5
    assert bench.whole_job_rate(1, 10, 2, 4.0) == pytest.approx(5e-9)

"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1 agree
on the max-over-ranks time and the whole-job throughput (replicas only)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    el, value = bench.aggregate([3.0, 5.0][rank], 1000, world, dist, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, el, value))


def test_two_ranks_report_max_time_and_total_points():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, el, value in got:
        assert el == 5.0
        assert value == 2 * 1000 / 5.0


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(2.0, 500, 1) == (2.0, 250.0)

"""The N > 1 path of bench.py on CPU: two gloo ranks run as independent replicas; the timing
is the slowest rank's and the throughput counts every rank's units (weak scaling).  No
data-path collective exists; only the timing reduction crosses ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [3.0, 5.0][rank]          # rank 1 is the slow replica
    slowest = bench.max_over_ranks(local_ms, world, "cpu")
    rate = bench.aggregate_rate(1000, world, slowest / 1e3)
    dist.barrier()
    q.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5.0, 5.0]
    assert all(abs(r[2] - 2 * 1000 / 0.005) < 1e-6 for r in res)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.25, 1, "cpu") == 4.25
    assert bench.aggregate_rate(10, 1, 2.0) == 5.0

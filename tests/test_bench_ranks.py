"""bench.py's multi-rank aggregation on CPU: two gloo ranks, replicas with
different timings; every rank sees the slowest time and the whole-job rate."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    t, value = bench.aggregate_ranks(1.0 + rank, 10)  # rank 1 is slower
    q.put((rank, t, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, value in out:
        assert t == 2.0 and value == 2 * 10 / 2.0


def test_single_process_needs_no_collective():
    import bench

    assert bench.aggregate_ranks(4.0, 8) == (4.0, 2.0)

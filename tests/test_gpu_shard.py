"""One layout divided over several contexts (tsgne_shard_*), on one GPU.

Two and three processes, each with its own context on cuda:0, divide the
exact repulsion's tile-pair units and sum their int64 force accumulators and
per-unit Z partials through gloo (host staging): no kernel of one process
waits on another, the only exchange is the host collective between two
launches.  Because both sums are exact, every rank's gradient and layout
must equal a single context's bit for bit, and therefore the oracle within
the single context's tolerances (gradient 1e-4 relative L2, Z 1e-5, layout
after 10 iterations 1e-4).
"""

import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import paper_2310_11186_gb300 as pkg  # noqa: E402
import tsgne_synth as synth  # noqa: E402

N = 5003


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_11186_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    yield


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _inputs():
    g = synth.random_graph(N, 7.0, seed=31)
    labels = (np.arange(N) % 7).astype(np.int32)
    X = synth.block_embedding(labels, 16, seed=31)
    rp, col, P = oracle.build_P(N, g.row_ptr, g.col, X, 3.0)
    Ys = synth.spread_layout(labels, scale=20.0, seed=32)
    Y0 = synth.y_init(N, seed=33)
    return rp, col, P.astype(np.float32), Ys, Y0


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    from paper_2310_11186_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    torch.cuda.set_device(0)
    rp, col, P, Ys, Y0 = _inputs()
    with shard.ShardedLayout(perplexity=3.0) as lay:
        lay.set_P(rp, col, P)
        lay.init_Y(Ys)
        G, Z = lay.gradient(12.0)
    with shard.ShardedLayout(perplexity=3.0) as lay:
        lay.set_P(rp, col, P)
        lay.init_Y(Y0)
        lay.run(10)
        Y10 = lay.get_Y()
    q.put((rank, G, Z, Y10))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_layout_equals_one_context_and_the_oracle(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=600) for _ in range(ws)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    rp, col, P, Ys, Y0 = _inputs()
    with pkg.Layout(perplexity=3.0) as lay:
        lay.set_P(rp, col, P)
        lay.init_Y(Ys)
        G1, Z1 = lay.gradient(12.0)
        lay.init_Y(Y0)
        lay.run(10)
        Y1 = lay.get_Y()
    for rank, G, Z, Y10 in out:
        assert np.array_equal(G, G1) and Z == Z1, rank
        assert np.array_equal(Y10, Y1), rank
    oG, oZ = oracle.gradient(N, rp, col, P.astype(np.float64), Ys.astype(np.float64), 12.0)
    assert abs(Z1 - oZ) / oZ < 1e-5
    assert np.linalg.norm(G1 - oG) / np.linalg.norm(oG) < 1e-4
    oY, _, _ = oracle.optimize(N, rp, col, P.astype(np.float64), Y0, 10)
    assert np.linalg.norm(Y1 - oY) / np.linalg.norm(oY) < 1e-4


def test_shard_calls_check_their_arguments():
    rp, col, P, Ys, Y0 = _inputs()
    with pkg.Layout(perplexity=3.0) as lay:
        lay.set_P(rp, col, P)
        lay.init_Y(Ys)
        for bad in ((0, 0), (2, 2), (-1, 2)):
            with pytest.raises(pkg.TsgneError) as e:
                pkg.tsgne_shard_set(lay.ctx, *bad)
            assert e.value.status == 1
        with pytest.raises(pkg.TsgneError):  # nothing enqueued yet
            pkg.tsgne_shard_step_finish(lay.ctx)
        pkg.tsgne_shard_set(lay.ctx, 0, 1)
        U, u0, u1, acc, zunit = pkg.tsgne_shard_repulsion(lay.ctx)
        assert (u0, u1) == (0, U) and acc.count == 2 * N and zunit.count == U
        with pytest.raises(pkg.TsgneError):  # the previous share is not finished
            pkg.tsgne_shard_repulsion(lay.ctx)
        G, Z = pkg.tsgne_shard_gradient_finish(lay.ctx, 1.0)  # world 1: the whole pass
        G1, Z1 = lay.gradient(1.0)
        assert np.array_equal(G, G1) and Z == Z1
    with pkg.Layout(repulsion=1) as lt:
        with pytest.raises(pkg.TsgneError) as e:
            pkg.tsgne_shard_set(lt.ctx, 0, 2)
        assert e.value.status == 1

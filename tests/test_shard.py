"""The sharding plan of one layout over several ranks, on CPU (gloo).

The exact repulsion is divided by tile-pair units: rank r of w evaluates
units [U r / w, U (r + 1) / w) of the U = nt (nt + 1) / 2 pairs of tiles,
adds its forces into int64 fixed-point accumulators and its Z partials into
its slots of a per-unit array, and the ranks sum both arrays.  These tests
emulate the per-rank arithmetic in numpy (FP64 pair terms, the library's
fixed-point scale), run the exchange over two gloo ranks, and check:

* the plan covers every unit exactly once (any world size);
* after the exchange every rank holds the same accumulators, equal bit for
  bit to one process summing all units, whatever the split;
* decoded, they equal the exact oracle rows and Z (Eq. 4) within the
  fixed-point resolution and FP64 rounding;
* a rank that leaves between steps makes the other rank's next collective
  fail with an error instead of hanging (short process-group timeout).
"""

import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import tsgne_synth as synth  # noqa: E402
from paper_2310_11186_gb300 import shard  # noqa: E402

TILE = 256  # a small tile, so a few thousand points make many units


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _fix_shift(n):
    c = 0
    while (1 << c) < n:
        c += 1
    return 62 - c


def _unit_tiles(units, nt):
    """(a, b) of units in the library's order: diagonal d = b - a by diagonal."""
    ab = [(a, a + d) for d in range(nt) for a in range(nt - d)]
    assert len(ab) == units
    return ab


def _share(Y, u0, u1):
    """int64 accumulators (2 n) and per-unit Z partials (U) of units [u0, u1):
    each unit's FP64 partial of a point, scaled by 2^s and rounded, as the
    kernels add their FP32 partials."""
    n = Y.shape[0]
    nt = (n + TILE - 1) // TILE
    U = nt * (nt + 1) // 2
    scale = 2.0 ** _fix_shift(n)
    acc = np.zeros(2 * n, np.int64)
    zunit = np.zeros(U, np.float64)
    for u, (a, b) in enumerate(_unit_tiles(U, nt)):
        if not u0 <= u < u1:
            continue
        ia = np.arange(a * TILE, min(n, (a + 1) * TILE))
        ib = np.arange(b * TILE, min(n, (b + 1) * TILE))
        d = Y[ia, None, :] - Y[None, ib, :]
        w = 1.0 / (1.0 + (d * d).sum(-1))
        f = (w * w)[..., None] * d
        if a == b:
            np.fill_diagonal(w, 0.0)  # the kernel's w_ii = 1 terms are removed from Z at the end
            fi = f.sum(1)
            zunit[u] = w.sum()
        else:
            fi = f.sum(1)
            fj = -f.sum(0)
            zunit[u] = 2.0 * w.sum()
            acc[2 * ib] += np.rint(fj[:, 0] * scale).astype(np.int64)
            acc[2 * ib + 1] += np.rint(fj[:, 1] * scale).astype(np.int64)
        acc[2 * ia] += np.rint(fi[:, 0] * scale).astype(np.int64)
        acc[2 * ia + 1] += np.rint(fi[:, 1] * scale).astype(np.int64)
    return acc, zunit


@pytest.mark.parametrize("units", [1, 2, 3, 10, 43071])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_plan_covers_every_unit_once(units, world):
    seen = np.zeros(units, np.int64)
    sizes = []
    for r in range(world):
        u0, u1 = shard.unit_range(units, r, world)
        seen[u0:u1] += 1
        sizes.append(u1 - u0)
    assert (seen == 1).all()
    assert max(sizes) - min(sizes) <= 1
    assert shard.tile_units(300000, 1024) == 293 * 294 // 2


def _worker(rank, ws, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    Y = synth.spread_layout((np.arange(n) % 5).astype(np.int32), scale=6.0, seed=3).astype(np.float64)
    nt = (n + TILE - 1) // TILE
    U = nt * (nt + 1) // 2
    u0, u1 = shard.unit_range(U, rank, ws)
    acc, zunit = _share(Y, u0, u1)
    a = torch.from_numpy(acc)
    z = torch.from_numpy(zunit)
    shard.allreduce_sum_([a, z])
    q.put((rank, a.numpy().copy(), z.numpy().copy()))
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_single_process_bits_and_the_oracle():
    n = 2500
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    (_, a0, z0), (_, a1, z1) = out
    assert np.array_equal(a0, a1) and np.array_equal(z0, z1)
    Y = synth.spread_layout((np.arange(n) % 5).astype(np.int32), scale=6.0, seed=3).astype(np.float64)
    nt = (n + TILE - 1) // TILE
    U = nt * (nt + 1) // 2
    a_all, z_all = _share(Y, 0, U)
    assert np.array_equal(a0, a_all) and np.array_equal(z0, z_all)  # same bits as one process
    F = a0.reshape(n, 2).astype(np.float64) / 2.0 ** _fix_shift(n)
    Z = float(np.sum(z0))  # the library sums the unit partials in unit order
    Fe, zr = oracle.repulsion_all(Y)
    assert np.abs(F - Fe).max() <= 1e-12 * np.abs(Fe).max() + 2.0 ** -_fix_shift(n) * 2 * U
    assert abs(Z - zr.sum()) <= 1e-12 * zr.sum()


def _put_and_exit(q, item):
    q.put(item)
    q.close()
    q.join_thread()  # the item is in the pipe before the process ends
    os._exit(0)


def _leaver(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=datetime.timedelta(seconds=5))
    t = torch.ones(8, dtype=torch.int64)
    shard.allreduce_sum_([t])  # step 1: both ranks take part
    if rank == 1:
        _put_and_exit(q, (rank, "left"))  # leaves between steps, with nothing in flight
    try:
        shard.allreduce_sum_([t])  # step 2: the peer is gone
        _put_and_exit(q, (rank, "no error"))
    except Exception as e:  # noqa: BLE001
        _put_and_exit(q, (rank, f"error: {type(e).__name__}"))
    _put_and_exit(q, (rank, "done"))


def test_a_rank_that_leaves_makes_the_next_exchange_fail():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_leaver, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(60)
    assert res[1] == "left"
    assert res[0].startswith("error"), res[0]

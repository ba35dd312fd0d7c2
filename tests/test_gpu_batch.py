"""Batched layouts and the serving loop (GPU, through the C ABI).

A member of a batch must evolve exactly as it does alone: the batched kernels
keep every member's arithmetic (including reduction orders) independent of the
other members, so these comparisons are bit-exact.  The batch of one is also
compared with the single-layout context path at the same tile size.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2310_11186_gb300 as pkg  # noqa: E402
import tsgne_synth as synth  # noqa: E402
from paper_2310_11186_gb300 import serve  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_11186_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    yield


def _graphs(sizes, seed=0, d=16):
    out = []
    for k, n in enumerate(sizes):
        g = synth.sbm_zipf(n, max(2, n // 400), n * 3, zipf_s=0.0, rewire=0.1, seed=seed + k)
        X = synth.block_embedding(g.labels, d, seed=seed + k)
        Y0 = synth.y_init(n, seed=seed + k)
        out.append((g, X, Y0))
    return out


def _alone(g, X, Y0, tile, iters, perp=30.0):
    with pkg.Batch(tile_warps=tile, perplexity=perp) as b:
        mid = b.add(g.row_ptr, g.col, X, Y0)
        b.run(iters)
        Y, it = b.get_Y(mid)
    assert it == iters
    return Y


def test_batch_of_one_equals_context_path():
    (g, X, Y0), = _graphs([2000], seed=3)
    with pkg.Layout() as lay:
        lay.build_P(g.row_ptr, g.col, X)
        lay.init_Y(Y0)
        tile = lay.repulsion_shape()["block"] // 32
        lay.run(30)
        Yc = lay.get_Y()
    Yb = _alone(g, X, Y0, tile, 30)
    assert np.array_equal(Yb, Yc)


def test_hub_rows_batch_equals_context_and_mix():
    """A power-law graph whose hub rows hold thousands of entries (summed in
    1024-entry warp chunks): a batch of one equals the single-layout path bit
    for bit, and in a mix with graphs without hub rows every member still
    equals itself alone."""
    g, X = synth.rmat(12, 1 << 17, seed=5)
    Y0 = synth.y_init(g.n, seed=5)
    with pkg.Layout() as lay:
        lay.build_P(g.row_ptr, g.col, X)
        rp, _, _ = lay.get_P()
        assert np.diff(rp).max() > 2 * 1024  # rows of several chunks
        lay.init_Y(Y0)
        tile = lay.repulsion_shape()["block"] // 32
        lay.run(30)
        Yc = lay.get_Y()
    Yb = _alone(g, X, Y0, tile, 30)
    assert np.array_equal(Yb, Yc)
    others = _graphs([900, 2500], seed=77)
    with pkg.Batch(tile_warps=tile) as b:
        ids = [b.add(gg.row_ptr, gg.col, XX, YY) for gg, XX, YY in others]
        hid = b.add(g.row_ptr, g.col, X, Y0)
        b.run(30)
        Yh, _ = b.get_Y(hid)
        Yo = [b.get_Y(i)[0] for i in ids]
    assert np.array_equal(Yh, Yb)
    for (gg, XX, YY), Y in zip(others, Yo):
        assert np.array_equal(Y, _alone(gg, XX, YY, tile, 30))


@pytest.mark.parametrize("tile", [1, 2, 4])
def test_members_in_a_mix_equal_alone(tile):
    gs = _graphs([700, 2000, 3500, 5003], seed=10)
    late = _graphs([1200], seed=40)[0]
    with pkg.Batch(tile_warps=tile) as b:
        ids = [b.add(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
        b.run(10)
        late_id = b.add(late[0].row_ptr, late[0].col, late[1], late[2])  # joins at iteration 10
        b.run(15)
        assert b.size()["members"] == 5
        mixed = [b.get_Y(i) for i in ids]
        late_Y, late_it = b.get_Y(late_id)
    for (g, X, Y0), (Y, it) in zip(gs, mixed):
        assert it == 25
        assert np.array_equal(Y, _alone(g, X, Y0, tile, 25))
    assert late_it == 15
    assert np.array_equal(late_Y, _alone(*late, tile, 15))


def test_batch_shapes_and_their_autotuner():
    """Every shape of the batched pass (1, 2, 4 warps x 8, 16 i-points per
    lane) keeps members independent (a member alone equals it in a mix at
    that shape); the shape autotuner picks one of them, resets the members,
    and a later run equals a fresh batch set to the same shape."""
    gs = _graphs([2600, 900, 4100], seed=140)
    for w, ri in ((1, 8), (4, 8), (2, 16)):
        with pkg.Batch() as b:
            b.set_shape(w, ri)
            ids = [b.add(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
            b.run(12)
            mixed = [b.get_Y(i)[0] for i in ids]
        for (g, X, Y0), Ym in zip(gs, mixed):
            with pkg.Batch() as b1:
                b1.set_shape(w, ri)
                i = b1.add(g.row_ptr, g.col, X, Y0)
                b1.run(12)
                assert np.array_equal(b1.get_Y(i)[0], Ym)
    with pkg.Batch() as b:
        ids = [b.add(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
        chosen, ms = b.autotune_shapes(trial_iters=2)
        assert chosen in pkg.Batch.BATCH_SHAPES and b.shape() == chosen and len(ms) == 6
        b.run(12)
        tuned = [b.get_Y(i)[0] for i in ids]
    with pkg.Batch() as b:
        b.set_shape(*chosen)
        ids = [b.add(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
        b.run(12)
        assert all(np.array_equal(b.get_Y(i)[0], t) for i, t in zip(ids, tuned))


def test_remove_keeps_others_unchanged():
    gs = _graphs([900, 1500, 2600], seed=20)
    with pkg.Batch(tile_warps=2) as b:
        ids = [b.add(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
        b.run(8)
        b.remove(ids[1])
        b.run(12)
        Y0_, it0 = b.get_Y(ids[0])
        Y2_, it2 = b.get_Y(ids[2])
        with pytest.raises(pkg.TsgneError):
            b.get_Y(ids[1])
    assert it0 == it2 == 20
    assert np.array_equal(Y0_, _alone(*gs[0], 2, 20))
    assert np.array_equal(Y2_, _alone(*gs[2], 2, 20))


def test_batched_layout_matches_oracle_short_horizon():
    """A batch member after 10 iterations against the FP64 oracle (1e-4 rel L2)."""
    (g, X, Y0), = _graphs([1800], seed=30)
    Y = _alone(g, X, Y0, 1, 10)
    rp, col, P = oracle.build_P(g.n, g.row_ptr, g.col, X, 30.0)
    oY, _, _ = oracle.optimize(g.n, rp, col, P, Y0, 10)
    assert np.linalg.norm(Y - oY) / np.linalg.norm(oY) < 1e-4


def test_autotune_resets_and_caches():
    gs = _graphs([1000, 3000, 6000], seed=50)
    with pkg.Batch() as b:
        for g, X, Y0 in gs:
            b.add(g.row_ptr, g.col, X, Y0)
        chosen, times = b.autotune(trial_iters=2)
        assert chosen in (1, 2, 4) and all(t > 0 for t in times.values())
        assert b.size()["tile_warps"] == chosen
        assert b.cached_tile() == chosen
        Y, it = b.get_Y(0)
        assert it == 0 and np.array_equal(Y, gs[0][2])


def test_serving_results_equal_alone():
    """Requests arriving while others run are admitted between ticks; each
    result equals the same request run alone (same tile, same iterations)."""
    gs = _graphs([800, 2500, 1300, 4000, 600], seed=60)
    arrivals = [0.0, 0.0, 0.02, 0.05, 0.05]
    reqs = [serve.Request(k, a, g.row_ptr, g.col, X, Y0) for k, (a, (g, X, Y0)) in enumerate(zip(arrivals, gs))]
    srv = serve.LayoutServer(iters=40, tick_iters=10, tile_warps=2)
    try:
        summary = srv.serve(reqs)
    finally:
        srv.close()
    assert summary["layouts"] == 5 and summary["p99_s"] >= summary["p50_s"] > 0
    for r, (g, X, Y0) in zip(reqs, gs):
        assert r.meta["device_iterations"] == 40
        assert np.array_equal(r.Y, _alone(g, X, Y0, 2, 40))


def test_serving_respects_memory_budget():
    gs = _graphs([3000, 3000, 3000], seed=70)
    reqs = [serve.Request(k, 0.0, g.row_ptr, g.col, X, Y0) for k, (g, X, Y0) in enumerate(gs)]
    one = serve.estimate_bytes(3000, int(gs[0][0].row_ptr[-1]) * 2, 2)
    srv = serve.LayoutServer(iters=20, tick_iters=10, tile_warps=2, budget_bytes=int(one * 1.5))
    try:
        summary = srv.serve(reqs)
    finally:
        srv.close()
    # only one layout fits at a time: admissions are staggered
    adm = sorted(r.admitted for r in reqs)
    fin = sorted(r.finished for r in reqs)
    assert summary["layouts"] == 3
    assert adm[1] >= fin[0] - 1e-9 and adm[2] >= fin[1] - 1e-9


def test_srpt_runs_short_jobs_first_and_results_stay_exact():
    """With room for one layout per tick, shortest-remaining-work-first lets
    the small requests overtake a large one that arrived first; inactive
    members keep their state, so every result still equals its run alone."""
    gs = _graphs([6000, 700, 900], seed=80)
    reqs = [serve.Request(k, 0.0, g.row_ptr, g.col, X, Y0) for k, (g, X, Y0) in enumerate(gs)]
    srv = serve.LayoutServer(iters=30, tick_iters=10, tile_warps=2, policy="srpt", fill_pairs=1.0)
    try:
        srv.serve(reqs)
    finally:
        srv.close()
    assert reqs[1].finished < reqs[0].finished and reqs[2].finished < reqs[0].finished
    for r, (g, X, Y0) in zip(reqs, gs):
        assert np.array_equal(r.Y, _alone(g, X, Y0, 2, 30))


def _tree_alone(g, X, Y0, iters, theta=0.5):
    with pkg.Layout(repulsion=1, theta=theta) as lay:
        lay.build_P(g.row_ptr, g.col, X)
        lay.init_Y(Y0)
        lay.run(iters)
        return lay.get_Y()


def test_tree_members_equal_the_single_layout_tree_code():
    """Tree-code members (their trees built and walked on branches of the
    batched iteration) evolve exactly as the single-layout tree code does,
    alone and in a mix with exact members and other tree members."""
    gs = _graphs([5000, 2600, 1200, 7000], seed=100)
    ref = [_tree_alone(g, X, Y0, 30) for g, X, Y0 in gs]
    with pkg.Batch(tile_warps=2, repulsion=1, theta=0.5) as b:  # every member a tree member
        ids = [b.add(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
        b.run(30)
        for mid, Yr in zip(ids, ref):
            assert np.array_equal(b.get_Y(mid)[0], Yr)
    with pkg.Batch(tile_warps=2, theta=0.5) as b:  # a mix: 0 and 2 tree, 1 and 3 exact
        ids = [b.add(g.row_ptr, g.col, X, Y0, repulsion=1 - (k % 2)) for k, (g, X, Y0) in enumerate(gs)]
        b.run(30)
        assert np.array_equal(b.get_Y(ids[0])[0], ref[0]) and np.array_equal(b.get_Y(ids[2])[0], ref[2])
        for k in (1, 3):
            g, X, Y0 = gs[k]
            assert np.array_equal(b.get_Y(ids[k])[0], _alone(g, X, Y0, 2, 30))


def test_serving_with_tree_members_equals_alone():
    """Requests of at least tree_min_n points are served as tree-code
    members; every result equals the same request run alone with the same
    repulsion (the serial comparison runs them the same way)."""
    gs = _graphs([900, 6000, 2200, 5000], seed=110)
    reqs = [serve.Request(k, 0.0, g.row_ptr, g.col, X, Y0) for k, (g, X, Y0) in enumerate(gs)]
    srv = serve.LayoutServer(iters=40, tick_iters=10, tile_warps=2, tree_min_n=4000)
    try:
        summary = srv.serve(reqs)
    finally:
        srv.close()
    assert summary["layouts"] == 4
    for r, (g, X, Y0) in zip(reqs, gs):
        want = _tree_alone(g, X, Y0, 40) if g.n >= 4000 else _alone(g, X, Y0, 2, 40)
        assert np.array_equal(r.Y, want)


@pytest.mark.parametrize("aging", [0, 2])
def test_aging_bounds_how_long_a_large_request_waits(aging):
    """One layout per tick (fill_pairs = 1), four requests of 4 ticks each
    submitted together.  Shortest remaining work first runs the three small
    ones first, so without aging the large one has not advanced after 6
    ticks; with aging_ticks = 2 it is chosen once it has been left out twice,
    so it has advanced by then.  Results stay those of each request alone."""
    gs = _graphs([6000, 700, 900, 800], seed=120)
    with pkg.Server(iters=40, tick_iters=10, tile_warps=2, policy=1, fill_pairs=1.0, aging_ticks=aging) as srv:
        ids = [srv.submit(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
        for _ in range(6):
            srv.tick()
        big_iters = srv.status(ids[0])[1]
        if aging == 0:
            assert big_iters == 0
        else:
            assert big_iters >= 10
        while srv.usage()["resident"] or srv.usage()["queued"]:
            srv.tick()
        for i, (g, X, Y0) in zip(ids, gs):
            assert np.array_equal(srv.result(i), _alone(g, X, Y0, 2, 40))


def test_requests_are_prepared_while_others_run():
    """A request admitted while another is resident is built by the
    server's worker thread during the tick (it is reported queued until it
    is attached at a later tick); one cancelled while it is being prepared
    is discarded when it comes back and its bytes are returned; every
    finished result equals its run alone."""
    gs = _graphs([5000, 1200, 900], seed=130)
    with pkg.Server(iters=60, tick_iters=10, tile_warps=2) as srv:
        a = srv.submit(gs[0][0].row_ptr, gs[0][0].col, gs[0][1], gs[0][2])
        srv.tick()  # nothing resident yet: the tick waits for a's member, then runs it
        assert srv.status(a) == ("resident", 10)
        one = srv.usage()["used_bytes"]
        b = srv.submit(gs[1][0].row_ptr, gs[1][0].col, gs[1][1], gs[1][2])
        c = srv.submit(gs[2][0].row_ptr, gs[2][0].col, gs[2][1], gs[2][2])
        srv.tick()  # admits b and c (prepared by the worker) while a advances
        assert srv.status(a) == ("resident", 20)
        srv.cancel(c)  # being prepared or prepared, not yet attached
        while srv.usage()["resident"] or srv.usage()["queued"]:
            srv.tick()
        assert srv.usage()["used_bytes"] == 0 and one > 0
        for rid, (g, X, Y0) in ((a, gs[0]), (b, gs[1])):
            assert srv.status(rid) == ("done", 60)
            assert np.array_equal(srv.result(rid), _alone(g, X, Y0, 2, 60))
        with pytest.raises(pkg.TsgneError) as e:
            srv.result(c)
        assert e.value.status == 8


def test_server_cancel_and_bookkeeping():
    """Cancelling a resident and a queued request frees them at once and their
    results report CANCELLED; the others finish exactly as alone, and the
    server's memory account returns to zero."""
    gs = _graphs([1500, 1200, 900, 700], seed=90)
    one = serve.estimate_bytes(1500, int(gs[0][0].row_ptr[-1]) * 2, 2)
    with pkg.Server(iters=30, tick_iters=10, tile_warps=2, policy=0, budget_bytes=int(2.5 * one)) as srv:
        ids = [srv.submit(g.row_ptr, g.col, X, Y0) for g, X, Y0 in gs]
        assert all(srv.status(i) == ("queued", 0) for i in ids)
        resident, queued, retired = srv.tick()
        assert resident == 2 and queued == 2 and retired == 0  # the budget holds two
        assert srv.status(ids[0]) == ("resident", 10)
        before = srv.usage()["used_bytes"]
        srv.cancel(ids[1])  # resident
        srv.cancel(ids[3])  # queued
        assert srv.usage()["used_bytes"] < before and srv.usage()["queued"] == 1
        with pytest.raises(pkg.TsgneError) as e:
            srv.cancel(ids[1])
        assert e.value.status == 1
        with pytest.raises(pkg.TsgneError) as e:
            srv.result(ids[0])  # not finished
        assert e.value.status == 5
        while srv.usage()["resident"] or srv.usage()["queued"]:
            srv.tick()
        assert sorted(srv.finished()) == [ids[0], ids[2]]
        for k in (0, 2):
            g, X, Y0 = gs[k]
            assert srv.status(ids[k]) == ("done", 30)
            assert np.array_equal(srv.result(ids[k]), _alone(g, X, Y0, 2, 30))
        for k in (1, 3):
            with pytest.raises(pkg.TsgneError) as e:
                srv.result(ids[k])
            assert e.value.status == 8
        assert srv.usage() == {"used_bytes": 0, "resident": 0, "queued": 0}

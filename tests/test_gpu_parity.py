"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: CSR structure bit-exact; P within 1e-5 relative per entry (the
per-row bisection runs in FP64 on both sides and p is rounded to FP32 once);
gradient at a fixed layout within 1e-4 relative L2 (FP32 with FP64 Z); Z and
KL at a fixed layout within 1e-5 relative; KL after a fixed seed and 1,000
iterations within 1e-3 relative; the layout after 10 iterations within 1e-4
relative L2.
"""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
import paper_2310_11186_gb300 as pkg  # noqa: E402
import tsgne_synth as synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_11186_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    yield


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _rand_csr(n, m, seed, hub=None, hub_deg=0):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    if hub is not None:
        src = np.concatenate([src, np.full(hub_deg, hub)])
        dst = np.concatenate([dst, rng.integers(0, n, hub_deg)])
    src = np.concatenate([src, src[: m // 5]])  # duplicates
    dst = np.concatenate([dst, dst[: m // 5]])
    perm = rng.permutation(src.size)
    src, dst = src[perm], dst[perm]
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    return np.cumsum(rp), dst.astype(np.int32)


# ------------------------------------------------------------- structure / P


@pytest.mark.parametrize(
    "n,m,seed,hub,hub_deg",
    [(2, 1, 0, None, 0), (50, 400, 1, None, 0), (3000, 20000, 2, 7, 3000), (20000, 60000, 3, 11, 9000)],
)
def test_structure_bit_exact(n, m, seed, hub, hub_deg):
    """Symmetric, sorted, unique, loop-free structure: all three sort tiers."""
    rp, col = _rand_csr(n, m, seed, hub, hub_deg)
    X = np.random.default_rng(seed).normal(size=(n, 4)).astype(np.float32)
    with pkg.Layout(perplexity=30.0) as lay:
        lay.build_P(rp, col, X)
        grp, gcol, gP = lay.get_P()
    orp, ocol = oracle.structure(n, rp, col)
    assert np.array_equal(grp, orp)
    assert np.array_equal(gcol, ocol)
    if hub is not None:
        assert np.diff(orp).max() > 4096 or n < 5000


@pytest.mark.parametrize("perp", [30.0, 2.0, 3.0, 5.0])
def test_P_matches_oracle_sbm2k(perp):
    g, X = synth.workload("sbm2k")
    with pkg.Layout(perplexity=perp) as lay:
        lay.build_P(g.row_ptr, g.col, X)
        rp, col, P = lay.get_P()
    orp, ocol, oP = oracle.build_P(g.n, g.row_ptr, g.col, X, perp)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    # relative bound, plus a floor far below any affinity that matters: at small
    # perplexities exp(-beta d) underflows (FP32 below ~1e-38 of the row maximum)
    tol = 1e-5 * oP + 1e-9 * oP.max()
    bad = np.abs(P - oP) > tol
    assert not bad.any(), f"{bad.sum()} entries, worst {np.max(np.abs(P - oP) / tol):.2f} x tol"
    assert abs(P.astype(np.float64).sum() - 1.0) < 1e-5


def test_P_device_pointers_match_host():
    g, X = synth.workload("sbm2k")
    with pkg.Layout(perplexity=5.0) as a, pkg.Layout(perplexity=5.0) as b:
        a.build_P(g.row_ptr, g.col, X)
        b.build_P(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(), torch.from_numpy(X).cuda())
        for x, y in zip(a.get_P(), b.get_P()):
            assert np.array_equal(x, y)


def test_bad_inputs_are_reported():
    X = np.zeros((3, 2), np.float32)
    with pkg.Layout() as lay:
        with pytest.raises(pkg.TsgneError) as e:
            lay.step()
        assert e.value.status == 5  # NOT_BUILT
        with pytest.raises(pkg.TsgneError) as e:
            lay.build_P(np.array([0, 2, 1, 2], np.int64), np.array([1, 2], np.int32), X)
        assert e.value.status == 2  # decreasing row_ptr
        with pytest.raises(pkg.TsgneError) as e:
            lay.build_P(np.array([0, 1, 2, 2], np.int64), np.array([1, 3], np.int32), X)
        assert e.value.status == 2  # column out of range
        with pytest.raises(pkg.TsgneError) as e:
            lay.build_P(np.array([1, 1, 2, 2], np.int64), np.array([1, 0], np.int32), X)
        assert e.value.status == 2  # row_ptr[0] != 0
        with pytest.raises(pkg.TsgneError) as e:
            lay.build_P(np.array([0, 1], np.int64), np.array([0], np.int32), X[:1])
        assert e.value.status == 1  # n < 2
        # the context is still usable
        lay.build_P(np.array([0, 1, 2, 2], np.int64), np.array([1, 0], np.int32), X)
        assert lay.sizes() == (3, 2)
    with pkg.Layout(perplexity=2.0) as lay:
        # star 0-{1,2,3}: row 0 has 3 > perplexity neighbours, so it bisects
        # on the distances, one of which is NaN
        star_rp = np.array([0, 3, 4, 5, 6], np.int64)
        star_col = np.array([1, 2, 3, 0, 0, 0], np.int32)
        Xn = np.zeros((4, 2), np.float32)
        Xn[2, 1] = np.nan
        with pytest.raises(pkg.TsgneError) as e:
            lay.build_P(star_rp, star_col, Xn)
        assert e.value.status == 6  # NONFINITE
        # the context is still usable
        lay.build_P(np.array([0, 1, 2, 2], np.int64), np.array([1, 0], np.int32), X)
        assert lay.sizes() == (3, 2)
        with pytest.raises(pkg.TsgneError) as e:
            lay.set_P(np.array([0, 1, 1, 1], np.int64), np.array([1], np.int32), np.array([1.0], np.float32))
        assert e.value.status == 2  # not symmetric


# ------------------------------------------------------------- gradient / Z


def _oracle_case(g, X, perp):
    rp, col, P = oracle.build_P(g.n, g.row_ptr, g.col, X, perp)
    return rp, col, P


@pytest.mark.parametrize(
    "n,deg,scale,alpha",
    [(3, 2.0, 1.0, 1.0), (37, 4.0, 2.0, 1.0), (2000, 10.0, 20.0, 1.0), (5003, 7.0, 20.0, 12.0),
     (5003, 7.0, 1e-4, 12.0), (9000, 6.0, 40.0, 1.0)],
)
def test_gradient_parity_fixed_Y(n, deg, scale, alpha):
    """g = 4 (alpha F^a - F^r / Z) at a fixed layout, oracle P installed with set_P;
    sizes span several i-blocks / j-tiles and ragged tails."""
    g = synth.random_graph(n, deg, seed=n)
    g.labels = (np.arange(n) % 7).astype(np.int32)
    X = synth.block_embedding(g.labels, 16, seed=n)
    rp, col, P = _oracle_case(g, X, 3.0)
    if scale < 1e-3:
        Y = synth.y_init(n, sigma=scale, seed=n)
    else:
        Y = synth.spread_layout(g.labels, scale=scale, seed=n)
    oG, oZ = oracle.gradient(n, rp, col, P, Y.astype(np.float64), alpha)
    with pkg.Layout() as lay:
        lay.set_P(rp, col, P.astype(np.float32))
        lay.init_Y(Y)
        G, Z = lay.gradient(alpha)
    assert abs(Z - oZ) / oZ < 1e-5, (Z, oZ)
    assert rel_l2(G, oG) < 1e-4, rel_l2(G, oG)
    # forces are pairwise antisymmetric: the gradient sums to ~0
    assert np.abs(G.astype(np.float64).sum(0)).max() < 1e-3 * np.abs(G).sum(0).max() + 1e-12


@pytest.mark.parametrize("sigma", [1e-3, 0.3])
def test_Z_in_a_tight_cloud(sigma):
    """The FP32 worst case for Z: 20,000 points in a cloud so tight that
    every term w is close to 1, so every FP32 partial grows with the number
    of its terms.  Partials of at most 64 terms, added in FP32 over at most
    16 groups and then in FP64, bound the relative rounding of Z by about
    (63 + 15) 2^-24 = 4.6e-6 in the worst case; random rounding keeps it far
    below that, and Z must agree with the oracle's FP64 sum within 1e-6."""
    n = 20000
    Y = synth.y_init(n, sigma=sigma, seed=17)
    _, zr = oracle.repulsion_all(Y.astype(np.float64))
    oZ = float(zr.sum())
    rp = np.zeros(n + 1, np.int64)
    with pkg.Layout() as lay:
        lay.set_P(rp, np.zeros(0, np.int32), np.zeros(0, np.float32))
        lay.init_Y(Y)
        _, Z = lay.gradient(1.0)
    assert abs(Z - oZ) / oZ < 1e-6, (Z, oZ, abs(Z - oZ) / oZ)


@pytest.mark.parametrize("shape", [(2, 16, 1), (1, 16, 1), (2, 8, 1), (1, 8, 1), (0, 0, 0)])
def test_every_repulsion_shape_matches_the_oracle(shape):
    """Each shape the autotuner can pick (symmetric with 1 or 2 warps and 8
    or 16 i-points per lane, or the ordered-pair kernel) gives the oracle's
    gradient and Z, and 10 iterations stay within the short-horizon bound."""
    n = 5003
    g = synth.random_graph(n, 6.0, seed=41)
    X = synth.block_embedding((np.arange(n) % 7).astype(np.int32), 16, seed=41)
    rp, col, P = _oracle_case(g, X, 3.0)
    Y = synth.spread_layout((np.arange(n) % 7).astype(np.int32), scale=20.0, seed=42)
    oG, oZ = oracle.gradient(n, rp, col, P, Y.astype(np.float64), 1.0)
    Y0 = synth.y_init(n, seed=43)
    oY, _, _ = oracle.optimize(n, rp, col, P, Y0, 10)
    with pkg.Layout() as lay:
        lay.set_P(rp, col, P.astype(np.float32))
        lay.set_repulsion_shape(*shape)
        lay.init_Y(Y)
        G, Z = lay.gradient(1.0)
        lay.init_Y(Y0)
        lay.run(10)
        Y10 = lay.get_Y()
    assert abs(Z - oZ) / oZ < 1e-5, (shape, Z, oZ)
    assert rel_l2(G, oG) < 1e-4, (shape, rel_l2(G, oG))
    assert rel_l2(Y10, oY) < 1e-4, (shape, rel_l2(Y10, oY))


def test_autotune_keeps_the_layout_and_picks_a_shape():
    g, X = synth.workload("sbm2k")
    Y0 = synth.y_init(g.n, seed=5)
    with pkg.Layout() as lay:
        lay.build_P(g.row_ptr, g.col, X)
        lay.init_Y(Y0)
        lay.run(4)
        Yb, Ub, Gb, itb = lay.get_state()
        chosen, ms = lay.autotune(2)
        Ya, Ua, Ga, ita = lay.get_state()
        assert np.array_equal(Ya, Yb) and np.array_equal(Ua, Ub) and ita == itb == 4
        assert chosen in pkg.Layout.REPULSION_SHAPES and min(v for v in ms.values() if v > 0) > 0
        lay.run(6)
        Yt = lay.get_Y()
    with pkg.Layout() as ref:  # the same shapes set by hand give the same bits
        ref.build_P(g.row_ptr, g.col, X)
        ref.init_Y(Y0)
        ref.run(4)  # the default shape, as before the autotuner ran
        ref.set_repulsion_shape(*chosen)
        ref.run(6)
        assert np.array_equal(ref.get_Y(), Yt)
    with pkg.Layout() as lay:
        lay.build_P(g.row_ptr, g.col, X)
        for bad in ((3, 16, 1), (2, 4, 1)):
            with pytest.raises(pkg.TsgneError):
                lay.set_repulsion_shape(*bad)
    with pkg.Layout(precision=1) as lay:  # the ordered kernel reads FP32 layouts only
        lay.build_P(g.row_ptr, g.col, X)
        with pytest.raises(pkg.TsgneError):
            lay.set_repulsion_shape(0, 0, False)


def test_gradient_two_nodes_vanishes():
    """2-node graph: p = q, the KL gradient is 0 for any layout."""
    with pkg.Layout() as lay:
        lay.set_P(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), np.array([0.5, 0.5], np.float32))
        lay.init_Y(np.array([[0.3, -1.0], [2.0, 0.5]], np.float32))
        G, Z = lay.gradient(1.0)
    assert np.abs(G).max() < 1e-6
    assert Z == pytest.approx(2.0 / (1 + 1.7 ** 2 + 1.5 ** 2), rel=1e-6)


def test_kl_parity_fixed_Y():
    g, X = synth.workload("sbm2k")
    rp, col, P = _oracle_case(g, X, 30.0)
    Y = synth.spread_layout(g.labels, scale=15.0)
    okl, oZ = oracle.kl(g.n, rp, col, P, Y.astype(np.float64))
    with pkg.Layout() as lay:
        lay.set_P(rp, col, P.astype(np.float32))
        lay.init_Y(Y)
        kl = lay.kl()
    assert abs(kl - okl) / okl < 1e-5, (kl, okl)


def test_isolated_and_edgeless_graphs():
    n = 700
    rp = np.zeros(n + 1, np.int64)
    X = np.zeros((n, 3), np.float32)
    Y = synth.spread_layout(np.zeros(n, np.int32), scale=1.0, jitter=3.0, seed=4)
    with pkg.Layout() as lay:
        lay.build_P(rp, np.zeros(0, np.int32), X)
        assert lay.sizes() == (n, 0)
        lay.init_Y(Y)
        G, Z = lay.gradient(1.0)
        assert lay.kl() == 0.0
    oG, oZ = oracle.gradient(n, rp, np.zeros(0, np.int32), np.zeros(0), Y.astype(np.float64), 1.0)
    assert rel_l2(G, oG) < 1e-4 and abs(Z - oZ) / oZ < 1e-5


# ---------------------------------------------------------------- iteration


def _sbm2k_gpu(perp=30.0, **cfg):
    g, X = synth.workload("sbm2k")
    lay = pkg.Layout(perplexity=perp, **cfg)
    lay.build_P(g.row_ptr, g.col, X)
    return g, X, lay


def test_layout_after_10_iterations():
    g, X, lay = _sbm2k_gpu()
    Y0 = synth.y_init(g.n)
    with lay:
        lay.init_Y(Y0)
        lay.run(10)
        Y = lay.get_Y()
    rp, col, P = _oracle_case(g, X, 30.0)
    oY, _, _ = oracle.optimize(g.n, rp, col, P, Y0, 10)
    assert rel_l2(Y, oY) < 1e-4, rel_l2(Y, oY)


def test_kl_after_1000_iterations_sbm2k():
    """The config the KL tolerance is stated on: 2,000-node SBM, seed 0,
    Y0 ~ N(0, 1e-4^2), 1,000 iterations, perplexity 30."""
    g, X, lay = _sbm2k_gpu()
    Y0 = synth.y_init(g.n)
    with lay:
        lay.init_Y(Y0)
        lay.run(1000)
        kl = lay.kl()
        Y = lay.get_Y()
    rp, col, P = _oracle_case(g, X, 30.0)
    oY, _, _ = oracle.optimize(g.n, rp, col, P, Y0, 1000)
    okl, _ = oracle.kl(g.n, rp, col, P, oY)
    assert abs(kl - okl) / okl < 1e-3, (kl, okl)
    assert np.all(np.isfinite(Y))


def test_run_equals_steps_and_is_deterministic():
    g, X, a = _sbm2k_gpu(perp=5.0)
    _, _, b = _sbm2k_gpu(perp=5.0)
    Y0 = synth.y_init(g.n, seed=3)
    with a, b:
        a.init_Y(Y0)
        b.init_Y(Y0)
        a.run(7)  # graph replay (3 x 2) + one direct step
        for _ in range(7):
            b.step()
        b.sync()
        assert np.array_equal(a.get_Y(), b.get_Y())
        a.run(6)
        b.run(6)
        assert np.array_equal(a.get_Y(), b.get_Y())


def test_checkpoint_resume_bit_identical():
    g, X, a = _sbm2k_gpu()
    _, _, b = _sbm2k_gpu()
    Y0 = synth.y_init(g.n, seed=5)
    with a, b:
        a.init_Y(Y0)
        a.run(300)  # crosses the end of early exaggeration (250)
        full = a.get_Y()
        b.init_Y(Y0)
        b.run(120)
        Y, U, G, it = b.get_state()
        assert it == 120
        b.close()
        with pkg.Layout() as c:
            c.build_P(g.row_ptr, g.col, X)
            c.set_state(Y, U, G, it)
            c.run(180)
            assert np.array_equal(c.get_Y(), full)


def test_nonfinite_layout_is_reported():
    g, X, lay = _sbm2k_gpu()
    Y = synth.spread_layout(g.labels)
    Y[5, 1] = np.inf
    with lay:
        lay.set_state(Y)
        with pytest.raises(pkg.TsgneError) as e:
            lay.run(2)
        assert e.value.status == 6


def test_device_layout_io():
    g, X, lay = _sbm2k_gpu()
    Y0 = torch.from_numpy(synth.y_init(g.n, seed=2)).cuda()
    with lay:
        lay.init_Y(Y0)
        lay.run(4)
        out = torch.empty((g.n, 2), dtype=torch.float32, device="cuda")
        lay.get_Y(out)
        assert np.array_equal(out.cpu().numpy(), lay.get_Y())
        G = torch.empty_like(out)
        lay.gradient(1.0, out=G)
        assert np.array_equal(G.cpu().numpy(), lay.gradient(1.0)[0])
        # device buffers of the wrong size never reach the library
        with pytest.raises(ValueError):
            lay.get_Y(torch.empty((g.n - 1, 2), dtype=torch.float32, device="cuda"))
        with pytest.raises(ValueError):
            lay.init_Y(Y0[:-1])
        with pytest.raises(ValueError):
            lay.set_state(Y0, update=torch.zeros((g.n, 1), dtype=torch.float32, device="cuda"))
        rp = torch.from_numpy(g.row_ptr).cuda()
        col = torch.from_numpy(g.col).cuda()
        with pytest.raises(ValueError):
            lay.build_P(rp, col[:-1], torch.from_numpy(X).cuda())
        with pytest.raises(ValueError):
            lay.build_P(rp, col, torch.from_numpy(X[:-1]).cuda())
        assert np.array_equal(out.cpu().numpy(), lay.get_Y())  # the layout is untouched


def test_gradient_parity_with_hub_rows():
    """Rows above 32 entries take the chunked path (one warp per 1,024-entry
    chunk, chunk sums added by the row's update thread)."""
    n = 6000
    rng = np.random.default_rng(3)
    g = synth.random_graph(n, 5.0, seed=77)
    hubs = {7: 3000, 4000: 800, 5999: 300}
    src, dst = [], []
    for h, k in hubs.items():
        nb = rng.choice(n, size=k, replace=False)
        nb = nb[nb != h]
        src.append(np.full(nb.size, h))
        dst.append(nb)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    rp, col = synth.csr_from_edges(n, np.concatenate([rows] + src), np.concatenate([g.col] + dst))
    labels = (np.arange(n) % 5).astype(np.int32)
    X = synth.block_embedding(labels, 8, seed=5)
    orp, ocol, oP = oracle.build_P(n, rp, col, X, 3.0)
    assert np.diff(orp).max() > 2000
    Y = synth.spread_layout(labels, scale=15.0, seed=9)
    for alpha in (1.0, 12.0):
        oG, oZ = oracle.gradient(n, orp, ocol, oP, Y.astype(np.float64), alpha)
        with pkg.Layout(perplexity=3.0) as lay:
            lay.build_P(rp, col, X)
            lay.init_Y(Y)
            G, Z = lay.gradient(alpha)
        assert rel_l2(G, oG) < 1e-4, rel_l2(G, oG)


@pytest.mark.parametrize("wl,k,perp", [("rand3000", 1, 2.0), ("rand3000", 5, 3.0), ("rand3000", 91, 30.0),
                                       ("sbm2k", 91, 30.0), ("sbm2k", 256, 30.0)])
def test_knn_neighbours_match_oracle(wl, k, perp):
    """k_nn > 0: BFS-k lists (Eq. 7) symmetrised by union; structure bit-exact,
    P within 1e-5 (at k = 91, perplexity 30 every row bisects)."""
    if wl == "sbm2k":
        g, X = synth.workload("sbm2k")
    else:
        g = synth.random_graph(3000, 6.0, seed=k)
        X = np.random.default_rng(k).normal(size=(3000, 12)).astype(np.float32)
    with pkg.Layout(perplexity=perp, k_nn=k) as lay:
        lay.build_P(g.row_ptr, g.col, X)
        rp, col, P = lay.get_P()
    orp, ocol = oracle.knn_structure(g.n, g.row_ptr, g.col, k)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    pc, _, _ = oracle.cond_affinity(g.n, orp, ocol, X, perp)
    oP, _ = oracle.joint_P(g.n, orp, ocol, pc)
    tol = 1e-5 * oP + 1e-9 * oP.max()
    assert not (np.abs(P - oP) > tol).any()


def test_device_memory_limit_gives_oom_and_recovers():
    """An allocation past the process-wide limit fails with OOM before any
    cudaMalloc; the context stays usable and, with the limit lifted, builds
    and computes exactly what a fresh context does."""
    g, X = synth.workload("sbm2k")
    Y0 = synth.y_init(g.n, seed=4)
    with pkg.Layout() as ref:
        ref.build_P(g.row_ptr, g.col, X)
        ref.init_Y(Y0)
        G0, Z0 = ref.gradient(1.0)
    base = pkg.device_memory_in_use()
    try:
        with pkg.Layout() as lay:
            pkg.set_device_memory_limit(pkg.device_memory_in_use() + 4096)
            with pytest.raises(pkg.TsgneError) as e:
                lay.build_P(g.row_ptr, g.col, X)
            assert e.value.status == 3
            pkg.set_device_memory_limit(0)
            lay.build_P(g.row_ptr, g.col, X)
            lay.init_Y(Y0)
            G, Z = lay.gradient(1.0)
            assert np.array_equal(G, G0) and Z == Z0
    finally:
        pkg.set_device_memory_limit(0)
    assert pkg.device_memory_in_use() == base


def test_layout_after_10_iterations_with_hub_rows():
    """The update path with rows above 32 entries (hub chunks and short rows
    in one launch, the hub rows updated by their last chunk) against the
    oracle's optimiser; also bit-identical from run to run."""
    n = 6000
    rng = np.random.default_rng(3)
    g = synth.random_graph(n, 5.0, seed=77)
    src, dst = [], []
    for h, k in {7: 3000, 4000: 800, 5999: 300, 100: 40}.items():
        nb = rng.choice(n, size=k, replace=False)
        nb = nb[nb != h]
        src.append(np.full(nb.size, h))
        dst.append(nb)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    rp, col = synth.csr_from_edges(n, np.concatenate([rows] + src), np.concatenate([g.col] + dst))
    labels = (np.arange(n) % 5).astype(np.int32)
    X = synth.block_embedding(labels, 8, seed=5)
    orp, ocol, oP = oracle.build_P(n, rp, col, X, 3.0)
    Y0 = synth.y_init(n, seed=9)
    oY, _, _ = oracle.optimize(n, orp, ocol, oP, Y0, 10)
    out = []
    for _ in range(2):
        with pkg.Layout(perplexity=3.0) as lay:
            lay.set_P(orp, ocol, oP.astype(np.float32))
            lay.init_Y(Y0)
            lay.run(10)
            out.append(lay.get_Y())
    assert np.array_equal(out[0], out[1])
    assert rel_l2(out[0], oY) < 1e-4, rel_l2(out[0], oY)


def test_exact_pass_size_limit_is_reported():
    """Above 2^24 - 2048 points the exact pass's tile-pair count would leave
    its 32-bit range: P builds, the layout is refused with INVALID_ARG and the
    context stays usable; a batch refuses such an exact member before any
    device work."""
    n = (1 << 24) - 2048 + 1
    rp = np.zeros(n + 1, np.int64)
    X = np.zeros((n, 1), np.float32)
    with pkg.Layout() as lay:
        with pytest.raises(pkg.TsgneError) as e:
            lay.build_P(rp, np.zeros(0, np.int32), X)
        assert e.value.status == 1
        lay.build_P(np.array([0, 1, 2, 2], np.int64), np.array([1, 0], np.int32), np.zeros((3, 2), np.float32))
        assert lay.sizes() == (3, 2)
    with pkg.Batch() as b:
        with pytest.raises(pkg.TsgneError) as e:
            b.add(rp, np.zeros(0, np.int32), X)
        assert e.value.status == 1

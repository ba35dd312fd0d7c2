"""Tree-code repulsion (cfg.repulsion = 1).

Parity reference: the EXACT sums of Eq. 4 (the oracle's plain O(n^2) rows),
under the error bound derived for the monopole approximation (the
second-order Taylor remainder of w and w^2 u about each accepted node's
centre of mass; derivation above ``node_bound`` in the oracle's C source),
which ``oracle.repulsion_tree_bounds`` evaluates per row.  Every checked row
must satisfy |F_gpu - F_exact| <= bound + 1e-4 A_i, with A_i the row's
absolute force sum (FP32 accumulation of at most a few thousand terms), and
Z must satisfy |Z_gpu - Z_exact| <= sum of the row bounds + 1e-5 Z.  This
runs on layouts of 2 ... 20,000 points (every row) and on the full 300K
benchmark graph (sampled rows, Z over all rows) at a spread layout and at the
layout after 1,000 iterations.

Determinism aid: the oracle also restates the tree code's own steps (same
FP32 decisions: keys, tree shape, acceptance), and the GPU's sums match
that restatement within the exact path's tolerances (gradient 1e-4 relative
L2, Z 1e-5); this shows both walk the same interactions, not that the
approximation is good -- the bound tests do that.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_11186_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    yield


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def grad_err(G, oG):
    """Relative L2 error; a gradient that vanishes (a 2-node graph has p = q)
    is compared in absolute terms instead."""
    nb = np.linalg.norm(oG)
    if nb < 1e-12:
        return float(np.abs(np.asarray(G, np.float64) - oG).max())
    return rel_l2(G, oG)


def _case(n, deg, seed, perp=3.0):
    g = synth.random_graph(n, deg, seed=seed)
    labels = (np.arange(n) % 7).astype(np.int32)
    X = synth.block_embedding(labels, 16, seed=seed)
    rp, col, P = oracle.build_P(n, g.row_ptr, g.col, X, perp)
    return labels, rp, col, P


def _layout(kind, labels, seed):
    n = labels.size
    if kind == "spread":
        return synth.spread_layout(labels, scale=20.0, seed=seed)
    if kind == "tiny":
        return synth.y_init(n, sigma=1e-4, seed=seed)
    if kind == "coincident":
        Y = synth.spread_layout(labels, scale=5.0, seed=seed)
        Y[: n // 3] = Y[0]  # a third of the points on one spot
        return Y
    raise ValueError(kind)


def _gpu_gradient(rp, col, P, Y, alpha, theta):
    with pkg.Layout(repulsion=1, theta=theta) as lay:
        lay.set_P(rp, col, P.astype(np.float32))
        lay.init_Y(Y)
        return lay.gradient(alpha)


@pytest.mark.parametrize("n,theta,kind", [
    (2, 0.5, "spread"), (33, 0.5, "spread"), (1000, 0.0, "spread"), (1000, 0.5, "spread"),
    (5003, 0.3, "spread"), (5003, 0.5, "tiny"), (5003, 1.0, "spread"), (9000, 0.5, "coincident"),
    (9000, 1.0, "coincident"), (20000, 0.5, "spread"),
])
def test_tree_gradient_matches_oracle_tree(n, theta, kind, record_property):
    labels, rp, col, P = _case(n, 6.0, seed=n)
    Y = _layout(kind, labels, seed=n)
    alpha = 12.0 if kind == "tiny" else 1.0
    oG, oZ = oracle.gradient_tree(n, rp, col, P, Y, alpha, theta=theta)
    G, Z = _gpu_gradient(rp, col, P, Y, alpha, theta)
    assert abs(Z - oZ) / oZ < 1e-5, (Z, oZ)
    assert grad_err(G, oG) < 1e-4, grad_err(G, oG)
    if n <= 5003 and n > 2:
        eG, eZ = oracle.gradient(n, rp, col, P, Y.astype(np.float64), alpha)
        record_property("grad_rel_l2_vs_exact", rel_l2(G, eG))
        record_property("Z_rel_vs_exact", abs(Z - eZ) / eZ)
        if theta == 0.0:
            assert rel_l2(G, eG) < 1e-4 and abs(Z - eZ) / eZ < 1e-5


def _gpu_repulsion(Y, theta):
    """F^r and Z of the tree code on the GPU: with no edges the gradient is
    g = -4 F^r / Z."""
    n = Y.shape[0]
    with pkg.Layout(repulsion=1, theta=theta) as lay:
        lay.set_P(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
        lay.init_Y(Y)
        G, Z = lay.gradient(1.0)
    return -G.astype(np.float64) * Z / 4.0, Z


def _abs_force_rows(Y, rows):
    """A_i = sum_{j != i} |w_ij^2 (y_i - y_j)| for the listed rows."""
    out = np.zeros(len(rows))
    for a in range(0, len(rows), 256):
        r = rows[a:a + 256]
        d = Y[r, None, :] - Y[None, :, :]
        r2 = (d * d).sum(-1)
        w = 1.0 / (1.0 + r2)
        out[a:a + 256] = (w * w * np.sqrt(r2)).sum(1)
    return out


def _check_within_bound(Y, theta, rows=None, Ze=None):
    """Checks the GPU tree code against the exact rows under the derived
    bound; returns (worst error / allowance over rows, Z error / allowance)."""
    Y = np.asarray(Y, np.float32).astype(np.float64)
    n = Y.shape[0]
    F, Z = _gpu_repulsion(Y, theta)
    _, _, _, bZ, bF = oracle.repulsion_tree_bounds(Y, theta)
    if rows is None:
        rows = np.arange(n)
        Fe, zre = oracle.repulsion_all(Y)
        Ze = float(zre.sum())
    else:
        Fe = np.concatenate([oracle.repulsion_rows(Y, int(i), int(i) + 1)[0] for i in rows])
    A = _abs_force_rows(Y, rows)
    err = np.linalg.norm(F[rows] - Fe, axis=1)
    allow = bF[rows].sum(1) + 1e-4 * A + 1e-30
    zallow = bZ.sum() + 1e-5 * Ze
    worst = float((err / allow).max())
    assert worst <= 1.0, (theta, rows[np.argmax(err / allow)], worst)
    assert abs(Z - Ze) <= zallow, (theta, Z, Ze, zallow)
    return worst, abs(Z - Ze) / zallow


@pytest.mark.parametrize("n,kind,theta", [
    (2, "spread", 0.5), (33, "spread", 0.8), (2000, "spread", 0.3), (2000, "spread", 1.0),
    (5003, "tiny", 0.5), (5003, "spread", 0.5), (9000, "coincident", 0.5), (9000, "coincident", 1.0),
    (20000, "spread", 0.3), (20000, "spread", 0.5), (20000, "spread", 0.8),
])
def test_tree_repulsion_within_derived_bound_of_exact(n, kind, theta, record_property):
    labels = (np.arange(n) % 7).astype(np.int32)
    Y = _layout(kind, labels, seed=n + 1)
    worst, zfrac = _check_within_bound(Y, theta)
    record_property("worst_err_over_allowance", worst)
    record_property("Z_err_over_allowance", zfrac)


def test_tree_far_clusters_monopole():
    """Two 32-point clusters 100 apart: each is one node for the other."""
    rng = np.random.default_rng(7)
    Y = np.concatenate([rng.uniform(-0.5, 0.5, size=(32, 2)),
                        rng.uniform(-0.5, 0.5, size=(32, 2)) + [100.0, 0.0]]).astype(np.float32)
    rp = np.zeros(65, np.int64)
    col = np.zeros(0, np.int32)
    P = np.zeros(0, np.float32)
    oG, oZ = oracle.gradient_tree(64, rp, col, P, Y, 1.0, theta=0.5)
    G, Z = _gpu_gradient(rp, col, P, Y, 1.0, 0.5)
    assert abs(Z - oZ) / oZ < 1e-6 and rel_l2(G, oG) < 1e-5


def test_tree_is_deterministic_and_iterates():
    """Bit-identical gradients, layouts and checkpoints from run to run."""
    g, X = synth.workload("sbm2k")
    Y0 = synth.y_init(g.n, seed=1)

    def run(k):
        lay = pkg.Layout(repulsion=1, theta=0.5)
        lay.build_P(g.row_ptr, g.col, X)
        lay.init_Y(Y0)
        lay.run(k)
        return lay

    a, b = run(300), run(300)
    with a, b:
        assert np.array_equal(a.get_Y(), b.get_Y())
        Ga, Za = a.gradient(1.0)
        Gb, Zb = b.gradient(1.0)
        assert np.array_equal(Ga, Gb) and Za == Zb
        c = run(120)
        Y, U, Gn, it = c.get_state()
        c.close()
        with pkg.Layout(repulsion=1, theta=0.5) as d:
            d.build_P(g.row_ptr, g.col, X)
            d.set_state(Y, U, Gn, it)
            d.run(180)
            assert np.array_equal(d.get_Y(), a.get_Y())


def test_tree_layout_quality(record_property):
    """1,000 iterations on the 2,000-node SBM: the final layouts of the exact
    path and of the tree code, both scored by the exact KL, differ by < 5%."""
    g, X = synth.workload("sbm2k")
    Y0 = synth.y_init(g.n, seed=0)
    finals = []
    for rep in (0, 1):
        with pkg.Layout(repulsion=rep, theta=0.5) as lay:
            lay.build_P(g.row_ptr, g.col, X)
            lay.init_Y(Y0)
            lay.run(1000)
            finals.append(lay.get_Y())
    assert all(np.all(np.isfinite(Yf)) for Yf in finals)
    kls = []
    with pkg.Layout() as ex:
        ex.build_P(g.row_ptr, g.col, X)
        for Yf in finals:
            ex.init_Y(Yf)
            kls.append(ex.kl())
    record_property("kl_exact", kls[0])
    record_property("kl_tree", kls[1])
    assert abs(kls[1] - kls[0]) / kls[0] < 5e-2, kls


def test_tree_full_size_zipf300k(record_property):
    """The benchmark's 300K-node workload at theta = 0.5 against the oracle's
    tree code on the same layout (all 300K rows)."""
    g, X = synth.workload("zipf300k")
    labels = g.labels
    Y = synth.spread_layout(labels, scale=30.0, seed=3)
    with pkg.Layout(repulsion=1, theta=0.5) as lay:
        lay.build_P(g.row_ptr, g.col, X)
        rp, col, P = lay.get_P()
        lay.init_Y(Y)
        G, Z = lay.gradient(1.0)
    oG, oZ = oracle.gradient_tree(g.n, rp, col, P.astype(np.float64), Y, 1.0, theta=0.5)
    record_property("grad_rel_l2", rel_l2(G, oG))
    assert abs(Z - oZ) / oZ < 1e-5, (Z, oZ)
    assert rel_l2(G, oG) < 1e-4, rel_l2(G, oG)


@pytest.mark.slow
def test_tree_full_size_zipf300k_within_derived_bound_of_exact(record_property):
    """The benchmark's 300K-node graph: the GPU tree code at theta = 0.3,
    0.5, 0.8 against the exact rows (sampled: hubs' endpoints, first, last,
    random) and the exact Z over all rows, each under the derived bound; at a
    spread layout and at the tree code's own layout after 1,000 iterations."""
    g, X = synth.workload("zipf300k")
    spread = synth.spread_layout(g.labels, scale=30.0, seed=3)
    with pkg.Layout(repulsion=1, theta=0.5) as lay:
        lay.build_P(g.row_ptr, g.col, X)
        lay.init_Y(synth.y_init(g.n, seed=0))
        lay.run(1000)
        late = lay.get_Y()
    rng = np.random.default_rng(5)
    deg = np.diff(g.row_ptr)
    rows = np.unique(np.concatenate([np.argsort(deg)[-8:], [0, g.n - 1], rng.choice(g.n, 240, replace=False)]))
    for name, Y in (("spread", spread), ("late", late)):
        Yd = np.asarray(Y, np.float32).astype(np.float64)
        _, zr = oracle.repulsion_all(Yd)
        Ze = float(zr.sum())
        for theta in (0.3, 0.5, 0.8):
            worst, zfrac = _check_within_bound(Yd, theta, rows=rows.astype(np.int32), Ze=Ze)
            record_property(f"{name}_theta{theta}_worst_err_over_allowance", worst)
            record_property(f"{name}_theta{theta}_Z_err_over_allowance", zfrac)


def test_tree_config_values():
    for bad in (dict(repulsion=2), dict(repulsion=1, theta=-0.1), dict(repulsion=1, theta=1.5)):
        with pytest.raises(pkg.TsgneError):
            pkg.Layout(**bad)
    for bad in (dict(repulsion=1, precision=1), dict(repulsion=1, theta=1.5)):
        with pytest.raises(pkg.TsgneError):
            pkg.Batch(**bad)
    with pkg.Batch(repulsion=1):  # tree-code members are allowed in batches
        pass


def test_tree_sort_wait_runs_out_and_recovers(record_property):
    """The sort's look-back waits are bounded by spin_budget_cycles.  With a
    budget of one cycle every wait that finds its predecessor tile not yet
    published gives up: that pass reports TSGNE_ERR_TIMEOUT (once) and the
    context stays usable.  Every pass that does not time out is bit-identical
    to the same pass with the default budget.  No GPU fault is involved: a
    wait that runs out returns normally."""
    g, X = synth.workload("zipf300k")
    Y = synth.spread_layout(g.labels, scale=30.0, seed=5)
    with pkg.Layout(repulsion=1, theta=0.5) as ref:
        ref.build_P(g.row_ptr, g.col, X)
        ref.init_Y(Y)
        G0, Z0 = ref.gradient(1.0)
    timeouts = 0
    with pkg.Layout(repulsion=1, theta=0.5, spin_budget_cycles=1) as lay:
        lay.build_P(g.row_ptr, g.col, X)
        lay.init_Y(Y)
        for _ in range(12):
            try:
                G, Z = lay.gradient(1.0)
            except pkg.TsgneError as e:
                assert e.name == "TSGNE_ERR_TIMEOUT", e
                timeouts += 1
                continue
            assert np.array_equal(G, G0) and Z == Z0
    record_property("timeouts_of_12", timeouts)
    with pytest.raises(pkg.TsgneError):
        pkg.Layout(repulsion=1, spin_budget_cycles=0)

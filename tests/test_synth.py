"""Seeded input generators: determinism and the stated workload shapes."""

import hashlib

import numpy as np

import tsgne_synth as synth


def _h(*arrs):
    h = hashlib.sha256()
    for a in arrs:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def test_counter_streams_are_consistent():
    a = synth.uniform(3, 1, 0, 100)
    b = synth.uniform(3, 1, 40, 60)
    assert np.array_equal(a[40:], b)
    z = synth.normal(3, 2, 0, 9)
    assert np.array_equal(z[3:], synth.normal(3, 2, 3, 6))
    assert not np.array_equal(synth.uniform(3, 1, 0, 10), synth.uniform(4, 1, 0, 10))
    x = synth.normal(0, 5, 0, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01


def test_sbm2k_shape_and_determinism():
    g, X = synth.workload("sbm2k")
    g2, X2 = synth.workload("sbm2k")
    assert _h(g.row_ptr, g.col, X) == _h(g2.row_ptr, g2.col, X2)
    e = g.m // 2
    assert abs(e - 10850) < 4 * np.sqrt(10850)  # 9950 intra + 900 inter expected
    assert X.shape == (2000, 128) and X.dtype == np.float32
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    assert np.all(g.col != rows)
    assert np.bincount(g.labels).tolist() == [200] * 10


def test_zipf_sizes_and_rewiring():
    sizes = synth.zipf_sizes(300_000, 50, 1.2)
    assert sizes.sum() == 300_000 and sizes[0] > sizes[-1]
    g = synth.sbm_zipf(20_000, 12, 60_000, 1.2, 0.10, seed=1)
    assert abs(g.m // 2 - 60_000) < 60
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    inter = np.mean(g.labels[rows] != g.labels[g.col])
    assert 0.05 < inter < 0.11  # ~10 % rewired, most to another block
    # simple graph: symmetric, no loops, no duplicates
    keys = rows.astype(np.int64) * g.n + g.col
    assert np.unique(keys).size == keys.size and np.all(rows != g.col)
    tkeys = np.sort(g.col.astype(np.int64) * g.n + rows)
    assert np.array_equal(np.sort(keys), tkeys)


# ------------------------------------------------- R-MAT (the precision-at-scale workload)


def _rmat_pairs(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return rows, g.col.astype(np.int64)


def test_rmat_edges_are_distinct_undirected_and_loop_free():
    g, X = synth.rmat(10, 5000, seed=3, chunk=1 << 15)
    u, v = _rmat_pairs(g)
    assert g.n == 1 << 10 and X.shape == (g.n, 64)
    assert g.row_ptr[-1] == 2 * 5000  # each edge in both directions
    assert not np.any(u == v)
    pairs = set(zip(u.tolist(), v.tolist()))
    assert len(pairs) == u.size  # no duplicate entries
    assert all((b, a) in pairs for a, b in pairs)


def test_rmat_quadrant_shares_follow_the_probabilities():
    """a = 0.57 for the (low, low) quadrant, d = 0.05 for (high, high), b + c =
    0.38 across; duplicates are dropped most in the dense quadrant, so its
    share sits a little below a.  A swapped probability moves a share far out."""
    g, _ = synth.rmat(12, 20000, seed=4, chunk=1 << 16)
    u, v = _rmat_pairs(g)
    h = g.n // 2
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    q00 = np.mean((lo < h) & (hi < h))
    q11 = np.mean((lo >= h) & (hi >= h))
    assert 0.45 < q00 < 0.60
    assert 0.03 < q11 < 0.08
    assert 0.33 < 1 - q00 - q11 < 0.48


def test_rmat_is_skewed_deterministic_and_has_64_communities():
    g, X = synth.rmat(11, 8000, seed=5, chunk=1 << 15)
    deg = np.diff(g.row_ptr)
    assert deg.max() > 10 * deg.mean()
    g2, X2 = synth.rmat(11, 8000, seed=5, chunk=1 << 15)
    assert np.array_equal(g.row_ptr, g2.row_ptr) and np.array_equal(g.col, g2.col) and np.array_equal(X, X2)
    g3, _ = synth.rmat(11, 8000, seed=6, chunk=1 << 15)
    assert not (np.array_equal(g.row_ptr, g3.row_ptr) and np.array_equal(g.col, g3.col))
    assert np.array_equal(g.labels, np.arange(g.n) >> (11 - 6)) and g.labels.max() == 63
    # the embedding clusters by community: a point is nearer its own community's mean
    means = np.stack([X[g.labels == c].mean(0) for c in range(64)])
    d_own = np.linalg.norm(X - means[g.labels], axis=1).mean()
    d_other = np.linalg.norm(X - means[(g.labels + 1) % 64], axis=1).mean()
    assert d_own < d_other


def test_induced_bfs_ball_is_a_bfs_prefix_with_its_induced_edges():
    g, _ = synth.rmat(10, 3000, seed=7, chunk=1 << 15)
    nodes, sub = synth.induced_bfs_ball(g, 300)
    assert nodes.size == 300 and np.unique(nodes).size == 300
    deg = np.diff(g.row_ptr)
    assert nodes[0] == np.argmax(deg)
    adj = [set(g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist()) for i in range(g.n)]
    pos = {int(x): k for k, x in enumerate(nodes)}
    for k in range(1, nodes.size):  # every node after the first hangs off an earlier one
        assert any(pos.get(w, 10**9) < k for w in adj[int(nodes[k])])
    want = {(pos[a], pos[b]) for a in pos for b in adj[a] if b in pos}
    u, v = _rmat_pairs(sub)
    assert set(zip(u.tolist(), v.tolist())) == want
    assert np.array_equal(sub.labels, g.labels[nodes])


def test_mixed_batch_respects_its_ranges():
    out = synth.sbm_mixed_batch(40, 500, 5000, 4.0, 12.0, 5, 40, 16, seed=2)
    ns = np.array([g.n for g, _ in out])
    assert ns.min() >= 500 and ns.max() <= 5000
    for g, X in out:
        mean_deg = g.row_ptr[-1] / g.n
        assert 3.5 <= mean_deg <= 12.5  # edges = round(n deg / 2), both directions stored
        assert X.shape == (g.n, 16)
        assert 1 <= g.labels.max() + 1 <= 40

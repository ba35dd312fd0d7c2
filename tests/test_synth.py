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

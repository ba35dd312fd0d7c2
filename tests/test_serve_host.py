"""Host-side pieces of the serving loop and the trace generators (CPU only)."""

import numpy as np

import tsgne_synth as synth
from paper_2310_11186_gb300 import serve


def test_estimate_bytes_grows_with_size_and_tile():
    a = serve.estimate_bytes(1000, 6000, 2)
    b = serve.estimate_bytes(10000, 60000, 2)
    assert b > a > 0
    # the repulsion slots scale as n^2 / tile: a smaller tile costs more memory
    assert serve.estimate_bytes(50000, 300000, 1) > serve.estimate_bytes(50000, 300000, 4)


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(20000, 20.0, seed=1)
    gaps = np.diff(t)
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 20.0) < 0.002
    assert abs(gaps.std() - 1 / 20.0) < 0.003  # exponential: std = mean


def test_log_uniform_sizes():
    n = synth.log_uniform_ints(50000, 1000, 300000, seed=2)
    assert n.min() >= 1000 and n.max() <= 300000
    # log-uniform: the median sits near the geometric mean of the bounds
    assert abs(np.log(np.median(n)) - 0.5 * (np.log(1000) + np.log(300000))) < 0.05


def test_summary_percentiles():
    reqs = []
    for k, lat in enumerate([1.0, 2.0, 3.0, 4.0]):
        r = serve.Request(k, 0.5, np.zeros(3, np.int64), np.zeros(0, np.int32), np.zeros((2, 2), np.float32))
        r.finished = 0.5 + lat
        reqs.append(r)
    s = serve.summarize(reqs, 10.0)
    assert s["layouts"] == 4 and s["p50_s"] == 2.5 and abs(s["layouts_per_s"] - 0.4) < 1e-12


def test_estimate_bytes_bounds_the_hub_row_chunks():
    """The estimate carries an upper bound for the hub-row chunk lists: it
    grows with nnz at a fixed n (a denser graph can hold more hub rows)."""
    a = serve.estimate_bytes(4096, 1 << 15, 1)
    b = serve.estimate_bytes(4096, 1 << 18, 1)
    assert b - a >= 8 * ((1 << 18) - (1 << 15))  # col + P at least

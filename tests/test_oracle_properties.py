"""Randomised pins for the FP64 oracle (CPU only, property-based).

The fixed cases of test_oracle.py, widened over random small inputs: graphs
with isolated nodes, duplicated edges and self-loops, n from 2 to 20,
random embeddings and layouts.  Every property is fixed by a definition of
the paper (Eqs. 2-5, 7) or by calculus, not by the oracle itself:

* N(i) is the symmetrised, loop-free union of the input edges (Eq. 7);
* P is non-negative, symmetric and sums to 1 (Eq. 3);
* KL equals the dense formula sum p ln(p / q), q = w / Z over all ordered
  pairs i != j (Eq. 5), and is >= 0;
* the gradient is the derivative of KL (central differences) and sums to
  zero over the points (pairwise antisymmetric forces);
* the tree code with theta = 0 sums every pair exactly (on a layout
  representable in FP32, the precision in which it takes the layout).
"""

import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle  # noqa: E402


def _csr_from_edges(n, edges):
    src = np.array([e[0] for e in edges], np.int64)
    dst = np.array([e[1] for e in edges], np.int32)
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    return np.cumsum(rp), dst


@st.composite
def graphs(draw, max_n=20):
    n = draw(st.integers(2, max_n))
    edges = draw(st.lists(st.tuples(st.integers(0, n - 1), st.integers(0, n - 1)), max_size=4 * n))
    seed = draw(st.integers(0, 2**31 - 1))
    return n, edges, seed


def _case(n, edges, seed, perp):
    rng = np.random.default_rng(seed)
    rp_in, col_in = _csr_from_edges(n, edges)
    X = rng.normal(size=(n, 3))
    rp, col, P = oracle.build_P(n, rp_in, col_in, X, perp)
    Y = rng.normal(scale=2.0, size=(n, 2))
    return rp_in, col_in, rp, col, P, Y


@settings(max_examples=60, deadline=None)
@given(graphs())
def test_structure_is_the_symmetrised_union(g):
    n, edges, _ = g
    rp_in, col_in = _csr_from_edges(n, edges)
    rp, col = oracle.structure(n, rp_in, col_in)
    want = [sorted({j for (a, b) in edges for (i2, j) in ((a, b), (b, a)) if i2 == i and j != i}) for i in range(n)]
    for i in range(n):
        assert list(col[rp[i]:rp[i + 1]]) == want[i]


@settings(max_examples=60, deadline=None)
@given(graphs(), st.sampled_from([2.0, 3.0, 5.0, 30.0]))
def test_P_is_symmetric_nonnegative_and_sums_to_one(g, perp):
    n, edges, seed = g
    _, _, rp, col, P, _ = _case(n, edges, seed, perp)
    assert np.all(P >= 0)
    if col.size:
        assert P.sum() == pytest.approx(1.0, rel=1e-12)
    D = {}
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            D[(i, int(col[e]))] = P[e]
    for (i, j), v in D.items():
        assert D[(j, i)] == pytest.approx(v, rel=1e-12, abs=1e-300)


@settings(max_examples=60, deadline=None)
@given(graphs())
def test_kl_is_the_dense_definition_and_nonnegative(g):
    n, edges, seed = g
    _, _, rp, col, P, Y = _case(n, edges, seed, 3.0)
    D2 = ((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    W = 1.0 / (1.0 + D2)
    np.fill_diagonal(W, 0.0)
    Q = W / W.sum()
    rows = np.repeat(np.arange(n), np.diff(rp))
    m = P > 0
    want = float((P[m] * np.log(P[m] / Q[rows[m], col[m]])).sum())
    v, z = oracle.kl(n, rp, col, P, Y)
    assert z == pytest.approx(W.sum(), rel=1e-12)
    assert v == pytest.approx(want, rel=1e-10, abs=1e-12)
    assert v >= -1e-12


@settings(max_examples=40, deadline=None)
@given(graphs(max_n=12))
def test_gradient_is_the_derivative_of_kl_and_sums_to_zero(g):
    n, edges, seed = g
    _, _, rp, col, P, Y = _case(n, edges, seed, 3.0)
    G, _ = oracle.gradient(n, rp, col, P, Y, 1.0)
    scale = np.abs(G).sum() + 1e-300
    assert np.abs(G.sum(0)).max() <= 1e-12 * scale + 1e-300
    FD = np.zeros_like(Y)  # without affinities the objective is ln Z (P = 0)
    for i in range(n):
        for c in range(2):
            h = 1e-6 * max(1.0, abs(Y[i, c]))
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, c] += h
            Ym[i, c] -= h
            fp = oracle.kl(n, rp, col, P, Yp)[0] if col.size else math.log(oracle.Z(Yp))
            fm = oracle.kl(n, rp, col, P, Ym)[0] if col.size else math.log(oracle.Z(Ym))
            FD[i, c] = (fp - fm) / (2 * h)
    assert np.linalg.norm(G - FD) <= 1e-5 * np.linalg.norm(FD) + 1e-9


@settings(max_examples=40, deadline=None)
@given(graphs(max_n=20), st.sampled_from([1.0, 12.0]))
def test_tree_code_at_theta_zero_is_exact(g, alpha):
    n, edges, seed = g
    _, _, rp, col, P, Y = _case(n, edges, seed, 3.0)
    Y = Y.astype(np.float32).astype(np.float64)  # the tree code takes the layout in FP32, as the GPU holds it
    G, Z = oracle.gradient(n, rp, col, P, Y, alpha)
    Gt, Zt = oracle.gradient_tree(n, rp, col, P, Y, alpha, theta=0.0)
    assert Zt == pytest.approx(Z, rel=1e-12)
    assert np.abs(Gt - G).max() <= 1e-12 * (np.abs(G).max() + 1e-300) + 1e-15

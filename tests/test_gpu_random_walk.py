"""Random-walk affinities (Eq. 6, cfg.p_walks > 0) against the oracle.

Both sides draw the same SplitMix64 numbers and take the same FP64
decisions, so the walk pairs (the structure of P) must match bit for bit and
P within 1e-6 relative (the joint normaliser is summed in another order,
then P is rounded to FP32).
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


def _check(n, row_ptr, col, X, R, L, seed, k_nn=0):
    if k_nn:
        rp0, col0 = oracle.knn_structure(n, row_ptr, col, k_nn)
    else:
        rp0, col0 = row_ptr, col
    orp, ocol, oP = oracle.random_walk_P(n, rp0, col0, X, R, L, seed)
    with pkg.Layout(p_walks=R, p_walk_length=L, seed=seed, k_nn=k_nn) as lay:
        lay.build_P(row_ptr, col, X.astype(np.float32))
        rp, cl, P = lay.get_P()
    assert np.array_equal(rp, orp) and np.array_equal(cl, ocol)
    assert np.all(np.abs(P - oP) <= 1e-6 * oP + 1e-12)
    return P


@pytest.mark.parametrize("n,deg,R,L", [(2, 1.0, 8, 1), (37, 3.0, 16, 2), (1000, 6.0, 64, 3), (3001, 8.0, 32, 5),
                                       (2000, 4.0, 512, 1)])
def test_random_walk_P_matches_oracle(n, deg, R, L):
    g = synth.random_graph(n, deg, seed=n + R)
    labels = (np.arange(n) % 5).astype(np.int32)
    X = synth.block_embedding(labels, 16, seed=n) * 0.25
    _check(n, g.row_ptr, g.col, X.astype(np.float32).astype(np.float64), R, L, seed=n)


def test_random_walk_with_hubs_isolated_nodes_and_knn():
    n = 4000
    g = synth.random_graph(n, 3.0, seed=3)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    hub = np.arange(1, 2500)
    src = np.concatenate([rows, np.zeros(hub.size, np.int64)])
    dst = np.concatenate([g.col, hub])
    keep = (src < 3900) & (dst < 3900)  # the last 100 nodes are isolated
    rp, col = synth.csr_from_edges(n, src[keep], dst[keep])
    X = synth.block_embedding((np.arange(n) % 4).astype(np.int32), 8, seed=2) * 0.3
    X = X.astype(np.float32).astype(np.float64)
    P = _check(n, rp, col, X, 24, 3, seed=7)
    assert P.sum() == pytest.approx(1.0, rel=1e-5)
    _check(600, *synth.csr_from_edges(600, np.arange(599), np.arange(1, 600)), X[:600], 16, 4, seed=1, k_nn=5)


def test_random_walk_layout_runs():
    g, X = synth.workload("sbm2k")
    with pkg.Layout(p_walks=64, p_walk_length=3) as lay:
        lay.build_P(g.row_ptr, g.col, X)
        lay.init_Y(synth.y_init(g.n, seed=0))
        lay.run(300)
        Y = lay.get_Y()
        assert np.all(np.isfinite(Y)) and lay.kl() > 0

"""ShortestPath embedding (Sec. 2.3, Eq. 8) on the GPU against the oracle: exact."""

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


def _targets(n, d, seed):
    return (synth.splitmix64(seed, 5, 0, d) % np.uint64(n)).astype(np.int32)


@pytest.mark.parametrize("n,deg,d,l0", [(2, 1.0, 1, 0), (500, 2.2, 5, 0), (3000, 6.0, 128, 0), (3000, 6.0, 100, 3),
                                        (20000, 8.0, 64, 0), (1200, 4.0, 300, 0)])
def test_shortest_path_exact(n, deg, d, l0):
    g = synth.random_graph(n, deg, seed=n + d)
    tg = _targets(n, d, seed=d)
    X = pkg.tsgne_shortest_path_embedding(g.row_ptr, g.col, tg, l0)
    srp, scol = oracle.structure(n, g.row_ptr, g.col)
    L0 = l0 if l0 > 0 else oracle.default_l0(scol.size // 2)
    oX = oracle.shortest_path_embedding(n, srp, scol, tg, L0)
    assert np.array_equal(X, oX.astype(np.float32))


def test_shortest_path_device_inputs_and_pipeline():
    g, _ = synth.workload("sbm2k")
    tg = _targets(g.n, 128, seed=1)
    Xh = pkg.tsgne_shortest_path_embedding(g.row_ptr, g.col, tg)
    Xd = pkg.tsgne_shortest_path_embedding(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(),
                                           torch.from_numpy(tg).cuda())
    assert np.array_equal(Xh, Xd.cpu().numpy())
    with pkg.Layout(perplexity=5.0) as a, pkg.Layout(perplexity=5.0) as b:
        a.build_P_shortest_path(g.row_ptr, g.col, tg)
        b.build_P(g.row_ptr, g.col, Xh)
        for x, y in zip(a.get_P(), b.get_P()):
            assert np.array_equal(x, y)


def test_shortest_path_rejects_bad_targets():
    g = synth.random_graph(50, 3.0, seed=1)
    with pytest.raises(pkg.TsgneError):
        pkg.tsgne_shortest_path_embedding(g.row_ptr, g.col, np.array([3, 50], np.int32))

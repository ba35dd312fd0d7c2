"""BF16 storage arm (precision = 1) against the FP64 oracle.

In this arm the force kernels read BF16 copies of P and of the layout and
compute in FP32 (Z and KL in FP64), so the exact result it approximates is
the oracle evaluated on the BF16-rounded P and Y; that comparison carries
the same tolerances as the FP32 arm (gradient 1e-4 relative L2, Z and KL
1e-5 relative).  The rounding is round-to-nearest-even to 8 significand
bits, done here by torch's CPU conversion.  The distance of the BF16 arm
from the unrounded oracle is a property of the format: it is recorded and
bounded only loosely, not a parity claim.
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


def bf16(a):
    """Round an FP32 array to BF16 (nearest even) and widen it to FP64."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_bf16_rounding_helper():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even significand wins (1)
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 1e30], np.float32)
    r = bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -6 and r[3] == -2.5
    assert abs(r[4] - 1e30) / 1e30 < 2.0 ** -8


@pytest.mark.parametrize("n,deg,scale,alpha", [(37, 4.0, 2.0, 1.0), (2000, 10.0, 20.0, 1.0),
                                                (5003, 7.0, 20.0, 12.0), (9000, 6.0, 40.0, 1.0)])
def test_bf16_gradient_equals_oracle_on_rounded_inputs(n, deg, scale, alpha, record_property):
    g = synth.random_graph(n, deg, seed=n)
    g.labels = (np.arange(n) % 7).astype(np.int32)
    X = synth.block_embedding(g.labels, 16, seed=n)
    rp, col, P = oracle.build_P(g.n, g.row_ptr, g.col, X, 3.0)
    P32 = P.astype(np.float32)
    Y = synth.spread_layout(g.labels, scale=scale, seed=n)
    oG, oZ = oracle.gradient(n, rp, col, bf16(P32), bf16(Y), alpha)
    with pkg.Layout(precision=1) as lay:
        lay.set_P(rp, col, P32)
        lay.init_Y(Y)
        G, Z = lay.gradient(alpha)
        # the getters return the FP32 master copies, not the BF16 shadows
        assert np.array_equal(lay.get_Y(), Y)
        assert np.array_equal(lay.get_P()[2], P32)
    assert abs(Z - oZ) / oZ < 1e-5, (Z, oZ)
    assert rel_l2(G, oG) < 1e-4, rel_l2(G, oG)
    # against the unrounded inputs the error is the format's: reported, and
    # only bounded loosely (coordinates of size ~20 carry a 2^-4 ulp, so
    # short edges lose most of their length's significant bits)
    fG, _ = oracle.gradient(n, rp, col, P, Y.astype(np.float64), alpha)
    record_property("bf16_grad_rel_l2_vs_fp64", rel_l2(G, fG))
    assert rel_l2(G, fG) < 0.5, rel_l2(G, fG)


def test_bf16_gradient_with_hub_rows():
    n = 6000
    rng = np.random.default_rng(3)
    g = synth.random_graph(n, 5.0, seed=77)
    src, dst = [], []
    for h, k in {7: 3000, 4000: 800, 5999: 300}.items():
        nb = rng.choice(n, size=k, replace=False)
        nb = nb[nb != h]
        src.append(np.full(nb.size, h))
        dst.append(nb)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    rp, col = synth.csr_from_edges(n, np.concatenate([rows] + src), np.concatenate([g.col] + dst))
    labels = (np.arange(n) % 5).astype(np.int32)
    X = synth.block_embedding(labels, 8, seed=5)
    orp, ocol, oP = oracle.build_P(n, rp, col, X, 3.0)
    Y = synth.spread_layout(labels, scale=15.0, seed=9)
    oG, oZ = oracle.gradient(n, orp, ocol, bf16(oP.astype(np.float32)), bf16(Y), 12.0)
    with pkg.Layout(perplexity=3.0, precision=1) as lay:
        lay.set_P(orp, ocol, oP.astype(np.float32))
        lay.init_Y(Y)
        G, Z = lay.gradient(12.0)
    assert abs(Z - oZ) / oZ < 1e-5
    assert rel_l2(G, oG) < 1e-4, rel_l2(G, oG)


def test_bf16_kl_equals_oracle_on_rounded_inputs():
    g, X = synth.workload("sbm2k")
    rp, col, P = oracle.build_P(g.n, g.row_ptr, g.col, X, 30.0)
    P32 = P.astype(np.float32)
    Y = synth.spread_layout(g.labels, scale=15.0)
    okl, _ = oracle.kl(g.n, rp, col, bf16(P32), bf16(Y))
    with pkg.Layout(precision=1) as lay:
        lay.set_P(rp, col, P32)
        lay.init_Y(Y)
        kl = lay.kl()
    assert abs(kl - okl) / okl < 1e-5, (kl, okl)


def _sbm2k(**cfg):
    g, X = synth.workload("sbm2k")
    lay = pkg.Layout(**cfg)
    lay.build_P(g.row_ptr, g.col, X)
    return g, X, lay


def test_bf16_layout_quality_and_determinism(record_property):
    """1,000 iterations from one seed: the BF16 arm is deterministic; its
    final KL is recorded beside the FP32 arm's and bounded loosely (the
    reads lose the short edges' lengths, so it ends a few percent higher)."""
    g, X, a = _sbm2k(precision=1)
    _, _, b = _sbm2k(precision=1)
    _, _, f = _sbm2k(precision=0)
    Y0 = synth.y_init(g.n, seed=0)
    with a, b, f:
        for lay in (a, b, f):
            lay.init_Y(Y0)
            lay.run(1000)
        Ya = a.get_Y()
        assert np.all(np.isfinite(Ya))
        assert np.array_equal(Ya, b.get_Y())
        kla, klf = a.kl(), f.kl()
    record_property("kl_bf16", kla)
    record_property("kl_fp32", klf)
    assert abs(kla - klf) / klf < 0.1, (kla, klf)


def test_bf16_checkpoint_resume_bit_identical():
    g, X, a = _sbm2k(precision=1)
    _, _, b = _sbm2k(precision=1)
    Y0 = synth.y_init(g.n, seed=5)
    with a, b:
        a.init_Y(Y0)
        a.run(300)
        full = a.get_Y()
        b.init_Y(Y0)
        b.run(120)
        Y, U, G, it = b.get_state()
        b.close()
        with pkg.Layout(precision=1) as c:
            c.build_P(g.row_ptr, g.col, X)
            c.set_state(Y, U, G, it)
            c.run(180)
            assert np.array_equal(c.get_Y(), full)


def test_precision_values():
    with pytest.raises(pkg.TsgneError):
        pkg.Layout(precision=2)
    with pytest.raises(pkg.TsgneError):
        pkg.Batch(precision=1)


def test_bf16_with_tree_code():
    """BF16 storage with the tree-code repulsion: the tree reads the FP32
    master layout (its keys and decisions are the FP32 tree's), the
    attraction reads the BF16 copies; deterministic, finite, and its
    gradient within the BF16 format error of the FP32 tree code's."""
    g, X = synth.workload("sbm2k")
    rp, col, P = oracle.build_P(g.n, g.row_ptr, g.col, X, 30.0)
    Y = synth.spread_layout(g.labels, scale=15.0)
    out = {}
    for prec in (0, 1):
        with pkg.Layout(precision=prec, repulsion=1, theta=0.5) as lay:
            lay.set_P(rp, col, P.astype(np.float32))
            lay.init_Y(Y)
            out[prec] = lay.gradient(1.0)
            lay.run(50)
            assert np.all(np.isfinite(lay.get_Y()))
    (G0, Z0), (G1, Z1) = out[0], out[1]
    assert Z1 == Z0  # the repulsion (and Z) come from the FP32 layout in both arms
    assert rel_l2(G1, G0.astype(np.float64)) < 0.5

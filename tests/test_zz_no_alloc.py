"""tsgne_repulsion_noalloc against the context-based repulsion.

The no-allocation entry point serves callers that cannot allocate device
memory themselves or through the library (a host framework owns the memory
budget, or an allocation would synchronise the device).  Its F^r and Z must
equal what the regular path computes: the regular path exports
g = 4 (alpha F^a - F^r / Z), so with alpha = 0, F^r = -g Z / 4.  Two calls in a
row, of different sizes, check that the shared scratch array carries nothing
over from one call to the next.  This file is collected last on purpose.

Sizes: 10,007 points is past the size where the pass caps its partial-force
chunks at the scratch array's limit and re-derives its grid; 65,536 is the
largest input the array is sized for.  Those two are checked against the
exact FP64 oracle directly; the small case runs last, so anything a larger
call left in the shared array would show up in it.
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


def _regular_path(n, Y, seed):
    g = synth.random_graph(n, 6.0, seed=seed)
    P = np.full(g.col.size, 1.0 / max(g.col.size, 1), np.float32)  # unused at alpha = 0
    with pkg.Layout() as lay:
        lay.set_P(g.row_ptr, g.col, P)
        lay.init_Y(Y)
        G, Z = lay.gradient(0.0)
    return -G.astype(np.float64) * Z / 4.0, Z


def _noalloc(Y):
    F, Z = pkg.tsgne_repulsion_noalloc(torch.from_numpy(Y).cuda())
    torch.cuda.synchronize()
    return F.cpu().numpy().astype(np.float64), float(Z.cpu().numpy()[0])


def test_noalloc_at_the_chunk_cap_and_the_maximum_against_the_oracle():
    for n, scale, seed in [(10007, 15.0, 21), (pkg.NOALLOC_MAX_N, 30.0, 22), (3001, 4.0, 23)]:
        labels = (np.arange(n) % 11).astype(np.int32)
        Y = synth.spread_layout(labels, scale=scale, seed=seed)
        F_ref, zr = oracle.repulsion_all(Y.astype(np.float64))
        Z_ref = float(zr.sum())
        F, Z = _noalloc(Y)
        assert abs(Z - Z_ref) / Z_ref < 1e-5, (n, Z, Z_ref)
        rel = np.linalg.norm(F - F_ref) / np.linalg.norm(F_ref)
        assert rel < 1e-4, (n, rel)


def test_noalloc_matches_regular_repulsion_twice():
    cases = [(5003, 20.0, 11), (1500, 3.0, 12)]
    for n, scale, seed in cases:
        labels = (np.arange(n) % 9).astype(np.int32)
        Y = synth.spread_layout(labels, scale=scale, seed=seed)
        F_ref, Z_ref = _regular_path(n, Y, seed)
        F, Z = pkg.tsgne_repulsion_noalloc(torch.from_numpy(Y).cuda())
        torch.cuda.synchronize()
        F = F.cpu().numpy().astype(np.float64)
        Z = float(Z.cpu().numpy()[0])
        assert abs(Z - Z_ref) / Z_ref < 1e-5, (n, Z, Z_ref)
        rel = np.linalg.norm(F - F_ref) / np.linalg.norm(F_ref)
        assert rel < 1e-4, (n, rel)


def test_noalloc_rejects_oversized_input():
    Y = torch.zeros((pkg.NOALLOC_MAX_N + 1, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.TsgneError) as e:
        pkg.tsgne_repulsion_noalloc(Y)
    assert e.value.status == 1 and "maximum" in str(e.value)


def test_noalloc_rejects_a_misaligned_layout():
    base = torch.zeros(2 * 1000 + 1, dtype=torch.float32, device="cuda")
    Y = base[1:].view(1000, 2)  # contiguous, but 4 bytes past an 8-byte boundary
    with pytest.raises(pkg.TsgneError) as e:
        pkg.tsgne_repulsion_noalloc(Y)
    assert e.value.status == 1 and "aligned" in str(e.value)

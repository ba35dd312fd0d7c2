"""The index-checking debug build (libtsgne_debug.so, -DTSGNE_DEBUG).

In the debug build every guarded device access first checks its index; a
failed check sets a bit of the context's status word, the access is
skipped (no trap, no out-of-bounds access) and the next synchronising call
returns TSGNE_ERR_INDEX.  Here the small-case parity suites run once more,
in a child process that loads the debug library (TSGNE_DEBUG=1): they must
pass as they do with the regular library, i.e. no check fires and every
result still matches the oracle.  A gradient through both libraries is also
compared: the checks do not change the arithmetic, so the bits agree.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import paper_2310_11186_gb300 as pkg, tsgne_synth as synth
assert pkg.library_path.endswith({libname!r}), pkg.library_path
g, X = synth.workload("sbm2k")
with pkg.Layout(perplexity=3.0) as lay:
    lay.build_P(g.row_ptr, g.col, X)
    lay.init_Y(synth.spread_layout(g.labels, scale=15.0, seed=2))
    G, Z = lay.gradient(12.0)
    lay.run(20)
    Y = lay.get_Y()
    kl = lay.kl()
with pkg.Layout(repulsion=1, theta=0.5) as lt:
    lt.build_P(g.row_ptr, g.col, X)
    lt.init_Y(synth.spread_layout(g.labels, scale=15.0, seed=2))
    Gt, Zt = lt.gradient(1.0)
np.savez({out!r}, G=G, Z=Z, Y=Y, kl=kl, Gt=Gt, Zt=Zt)
"""


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_11186_gb300 import build

    build.build()
    build.build(debug=True)
    yield


def _run(debug, out):
    env = dict(os.environ)
    env["TSGNE_DEBUG"] = "1" if debug else "0"
    code = CHILD.format(root=ROOT, out=str(out), libname="libtsgne_debug.so" if debug else "libtsgne.so")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_debug_build_gives_the_same_bits(tmp_path):
    a = _run(False, tmp_path / "regular.npz")
    b = _run(True, tmp_path / "debug.npz")
    for k in ("G", "Z", "Y", "kl", "Gt", "Zt"):
        assert np.array_equal(a[k], b[k]), k


def test_small_parity_suites_pass_under_the_debug_build():
    env = dict(os.environ)
    env["TSGNE_DEBUG"] = "1"
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_tree.py", "tests/test_gpu_bf16.py",
             "tests/test_gpu_batch.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu and not slow",
                        *files], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]

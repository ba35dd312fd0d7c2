"""The JSON-lines progress log (monitor.run_logged) on a real layout."""

import io
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2310_11186_gb300 as pkg  # noqa: E402
import tsgne_synth as synth  # noqa: E402
from paper_2310_11186_gb300 import monitor  # noqa: E402


def test_run_logged_writes_one_line_per_chunk_and_matches_a_plain_run():
    g, X = synth.workload("sbm2k")
    Y0 = synth.y_init(g.n, seed=6)
    buf = io.StringIO()
    with pkg.Layout(profile=1) as lay, pkg.Layout() as ref:
        for L in (lay, ref):
            L.build_P(g.row_ptr, g.col, X)
            L.init_Y(Y0)
        recs = monitor.run_logged(lay, 100, every=30, out=buf)
        ref.run(100)
        # logging (KL and gradient passes in between) does not change the layout
        assert np.array_equal(lay.get_Y(), ref.get_Y())
        assert lay.kl() == pytest.approx(recs[-1]["kl"], rel=1e-12)
    lines = [json.loads(l) for l in buf.getvalue().splitlines()]
    assert lines == recs and [r["iter"] for r in recs] == [30, 60, 90, 100]
    for r in recs:
        assert r["kl"] > 0 and r["grad_norm"] > 0 and r["iters_per_s"] > 0
        assert r["kernels_ms"]["repulsion"] > 0 and "attract_update" in r["kernels_ms"]

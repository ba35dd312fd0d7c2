"""The JSON line of `bench.py --impl reference` (the timed FP64 oracle arm),
run on CPU on the small block-model workload: one line, the keys the
benchmark contract names, and a value that is the fraction of an iteration
each step covers over the measured step time."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "sbm2k", "--steps", "2", "--warmup", "3",
           "--ref-step-seconds", "0.05"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, lines
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["unit"] == "iters/s" and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["workload"] == "sbm2k" and d["config"]["nodes"] == 2000
    assert d["value"] > 0 and d["ms_per_step"] > 0
    frac = d["iteration_fraction_per_step"]
    assert 0 < frac <= 1
    assert abs(d["value"] - frac / (d["ms_per_step"] / 1e3)) <= 1e-9 * d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0

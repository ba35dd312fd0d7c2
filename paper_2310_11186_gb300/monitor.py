"""Progress log of a layout as JSON lines.

``run_logged`` advances a ``Layout`` in chunks of ``every`` iterations and,
after each chunk, writes one JSON object per line: the iteration count, the
objective KL (Eq. 5), the gradient norm at the current layout, the
iterations per second of the chunk, and, when the layout was created with
``profile=1``, the device milliseconds per kernel class of the chunk.  The
KL and the gradient each cost one repulsion pass; every number comes from
the library's kernels through its C calls.
"""

from __future__ import annotations

import json
import sys
import time

import numpy as np

__all__ = ["run_logged"]


def run_logged(layout, n_iter: int, every: int = 50, out=None, grad: bool = True) -> list[dict]:
    """Runs n_iter iterations; returns the records it wrote to ``out``
    (default stdout; None-like objects without ``write`` are skipped)."""
    if every < 1:
        raise ValueError("every must be >= 1")
    out = sys.stdout if out is None else out
    records = []
    done = 0
    it0 = int(layout.get_state()[3])
    profiled = bool(getattr(layout, "config", None) is not None and layout.config.profile)
    if profiled:
        layout.kernel_times(reset=True)
    while done < n_iter:
        k = min(every, n_iter - done)
        t0 = time.perf_counter()
        layout.run(k)
        dt = time.perf_counter() - t0
        done += k
        rec = {"iter": it0 + done, "iters_per_s": k / dt if dt > 0 else None,
               "kl": float(layout.kl())}
        if grad:
            G, Z = layout.gradient(1.0)
            rec["grad_norm"] = float(np.linalg.norm(np.asarray(G, np.float64)))
            rec["Z"] = float(Z)
        if profiled:
            kt = layout.kernel_times(reset=True)
            rec["kernels_ms"] = {name: ms for name, (ms, launches) in kt.items() if launches}
        records.append(rec)
        if hasattr(out, "write"):
            out.write(json.dumps(rec) + "\n")
    return records

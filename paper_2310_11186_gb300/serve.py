"""Trace replay over the library's continuous-batching server.

Requests (a graph's CSR + embedding, optionally Y0) arrive over time.  The
scheduling itself -- the FIFO queue, admission while the estimated device
memory of the resident layouts stays within the budget and below the free
device memory, shortest-remaining-work-first selection, ticks of batched
iterations, retirement of finished layouts to host memory, cancellation --
runs in the library (``tsgne_server_*``, wrapped by ``Server``).  This
module only replays a trace in real time: it submits each request when its
arrival time has passed, calls ``tick`` and collects finished layouts, and
it measures latency from arrival to the layout being on the host.  Every
layout computation runs in the library's CUDA kernels; each request evolves
exactly as it would alone (same tile size).
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Server, server_estimate_bytes, tsgne_config_default

__all__ = ["Request", "LayoutServer", "estimate_bytes", "summarize", "serial_baseline"]


@dataclass
class Request:
    """One layout request; ``arrival`` is in seconds from the start of the trace."""

    rid: int
    arrival: float
    row_ptr: np.ndarray
    col: np.ndarray
    X: np.ndarray
    Y0: np.ndarray | None = None
    # filled in by the replay
    admitted: float | None = None
    finished: float | None = None
    Y: np.ndarray | None = None
    iterations: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


def estimate_bytes(n: int, nnz: int, tile_warps: int) -> int:
    """Device bytes a resident layout holds in a batch (the library's
    admission estimate, tsgne_server_estimate_bytes)."""
    return server_estimate_bytes(n, nnz, tile_warps)


class LayoutServer:
    """Policies: ``"all"`` advances every resident layout at every tick;
    ``"srpt"`` (shortest remaining processing time first) advances the
    resident layouts with the least remaining work (remaining iterations x
    n^2) until their pairs per iteration reach ``fill_pairs``; the others
    wait, resident, and a layout left out of ``aging_ticks`` ticks in a row
    goes first at the next tick (0: no aging).  Both run in the library.
    Requests of at least ``tree_min_n`` points (0: none) run the tree-code
    repulsion (the configuration's theta); the others the exact pass."""

    def __init__(self, iters: int = 500, tick_iters: int = 10, budget_bytes: int = 80 * 2 ** 30,
                 max_members: int = 256, tile_warps: int = 2, config=None, stream=None, policy: str = "srpt",
                 fill_pairs: float = 4e9, aging_ticks: int = 20, tree_min_n: int = 0):
        if policy not in ("all", "srpt"):
            raise ValueError("policy must be 'all' or 'srpt'")
        self.iters = iters
        self.tick_iters = tick_iters
        self.tile_warps = tile_warps
        self.config = config if config is not None else tsgne_config_default()
        self.server = Server(self.config, stream=stream, budget_bytes=int(budget_bytes), iters=int(iters),
                             tick_iters=int(tick_iters), max_members=int(max_members), tile_warps=int(tile_warps),
                             policy=1 if policy == "srpt" else 0, fill_pairs=float(fill_pairs),
                             aging_ticks=int(aging_ticks), tree_min_n=int(tree_min_n))
        self.ticks = 0

    def serve(self, requests: list[Request], clock=time.perf_counter) -> dict:
        """Replays a trace in real time; returns the summary (requests are updated in place)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        k = 0
        waiting: dict[int, Request] = {}  # submitted, not yet resident
        running: dict[int, Request] = {}
        done: list[Request] = []
        while k < len(pending) or waiting or running:
            now = clock() - t0
            while k < len(pending) and pending[k].arrival <= now:
                r = pending[k]
                rid = self.server.submit(r.row_ptr, r.col, r.X, r.Y0)
                r.meta["request_id"] = rid
                waiting[rid] = r
                k += 1
            if not waiting and not running:
                time.sleep(max(0.0, min(0.05, pending[k].arrival - (clock() - t0))))
                continue
            self.server.tick()
            self.ticks += 1
            now = clock() - t0
            for rid in list(waiting):
                if self.server.status(rid)[0] != "queued":
                    r = waiting.pop(rid)
                    r.admitted = now
                    running[rid] = r
            for rid in self.server.finished():
                r = running.pop(rid)
                r.iterations = self.server.status(rid)[1]
                r.meta["device_iterations"] = r.iterations
                r.Y = self.server.result(rid)
                r.finished = clock() - t0
                done.append(r)
        wall = clock() - t0
        return summarize(done, wall)

    def close(self):
        self.server.close()


def summarize(done: list[Request], wall: float) -> dict:
    lat = np.array([r.latency for r in done], dtype=np.float64)
    if lat.size == 0:
        return {"layouts": 0, "wall_s": wall}
    return {
        "layouts": int(lat.size),
        "wall_s": wall,
        "layouts_per_s": lat.size / wall,
        "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()),
        "max_s": float(lat.max()),
    }


def serial_baseline(requests: list[Request], iters: int, config=None, clock=time.perf_counter,
                    tree_min_n: int = 0) -> dict:
    """The same trace served one layout at a time (first come, first served)
    with the single-layout context API: the plain-run comparison point.
    Requests of at least ``tree_min_n`` points (0: none) run the tree code,
    as the server runs them, so both arms compute the same layouts."""
    import copy

    from . import Layout

    cfg = config if config is not None else tsgne_config_default()
    tcfg = copy.copy(cfg)
    tcfg.repulsion = 1
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    lats = []
    for r in pending:
        now = clock() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        with Layout(tcfg if (tree_min_n > 0 and r.n >= tree_min_n) else cfg) as lay:
            lay.build_P(r.row_ptr, r.col, r.X)
            lay.init_Y(r.Y0)
            lay.run(iters)
            lay.get_Y()
        lats.append(clock() - t0 - r.arrival)
    wall = clock() - t0
    lat = np.array(lats)
    return {"layouts": len(lats), "wall_s": wall, "layouts_per_s": len(lats) / wall,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}

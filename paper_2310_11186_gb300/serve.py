"""Continuous-batching layout server on top of the batch C ABI.

Requests (a graph's CSR + embedding, optionally Y0) arrive over time.  The
server keeps one ``Batch``: at every tick it admits the requests that have
arrived, as long as the estimated device memory of all resident layouts stays
within the budget (and below the free device memory), runs ``tick_iters``
iterations of every resident layout in one batched call, and retires the
layouts that reached ``iters`` iterations (their layout is copied to the host
and their device memory freed).  A request's latency runs from its arrival
to its layout being on the host.  The requests in flight overlap on the
device; each one evolves exactly as it would alone (same tile size), because
the batched kernels keep every member's arithmetic independent of the others.

All host-side scheduling lives here; every layout computation runs in the
library's CUDA kernels.
"""

from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import Batch, tsgne_config_default

__all__ = ["Request", "LayoutServer", "estimate_bytes"]


@dataclass
class Request:
    """One layout request; ``arrival`` is in seconds from the start of the trace."""

    rid: int
    arrival: float
    row_ptr: np.ndarray
    col: np.ndarray
    X: np.ndarray
    Y0: np.ndarray | None = None
    # filled in by the server
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
    """Device bytes a resident layout holds in a batch (P, layout, optimiser
    state, initial layout, per-tile repulsion slots and Z partials)."""
    T = 256 * tile_warps
    n_pad_max = -(-n // 2048) * 2048
    nt = -(-n // T)
    n_pad = nt * T
    units = nt * (nt + 1) // 2
    return (8 * (n + 1) + 8 * nnz + 5 * 8 * n_pad_max + 8 * n + 8 * nt * n_pad + 8 * units + 256)


class LayoutServer:
    """Policies: ``"all"`` advances every resident layout at every tick;
    ``"srpt"`` (shortest remaining processing time first) advances, at each
    tick, the resident layouts with the least remaining work (remaining
    iterations x n^2) until their pairs per iteration reach ``fill_pairs``
    (enough tile pairs to keep every SM busy), so small requests are not held
    behind large ones while the GPU stays full; the others wait, resident."""

    def __init__(self, iters: int = 500, tick_iters: int = 10, budget_bytes: int = 80 * 2 ** 30,
                 max_members: int = 256, tile_warps: int = 2, config=None, stream=None, policy: str = "srpt",
                 fill_pairs: float = 4e9):
        if iters % tick_iters != 0:
            raise ValueError("iters must be a multiple of tick_iters (layouts join and leave between ticks)")
        if policy not in ("all", "srpt"):
            raise ValueError("policy must be 'all' or 'srpt'")
        self.policy = policy
        self.fill_pairs = fill_pairs
        self.active: set[int] = set()
        self.iters = iters
        self.tick_iters = tick_iters
        self.budget = budget_bytes
        self.max_members = max_members
        self.tile_warps = tile_warps
        self.config = config if config is not None else tsgne_config_default()
        self.batch = Batch(self.config, tile_warps=tile_warps, stream=stream)
        self.resident: dict[int, tuple[Request, int]] = {}  # member id -> (request, bytes)
        self.used = 0
        self.ticks = 0

    def _free_device_bytes(self) -> int:
        try:
            import torch

            free, _ = torch.cuda.mem_get_info()
            return int(free)
        except Exception:  # pragma: no cover
            return self.budget

    def _admit(self, req: Request, now: float) -> bool:
        need = estimate_bytes(req.n, int(req.row_ptr[-1]) * 2, self.tile_warps)
        if self.resident and (len(self.resident) >= self.max_members or self.used + need > self.budget
                              or need > self._free_device_bytes()):
            return False
        mid = self.batch.add(req.row_ptr, req.col, req.X, req.Y0)
        self.active.add(mid)
        self.resident[mid] = (req, need)
        self.used += need
        req.admitted = now
        return True

    def serve(self, requests: list[Request], clock=time.perf_counter) -> dict:
        """Serves a trace in real time; returns the summary (requests are updated in place)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        k = 0
        waiting: list[Request] = []
        done: list[Request] = []
        while k < len(pending) or waiting or self.resident:
            now = clock() - t0
            while k < len(pending) and pending[k].arrival <= now:
                waiting.append(pending[k])
                k += 1
            while waiting and self._admit(waiting[0], now):
                waiting.pop(0)
            if not self.resident:
                if k < len(pending):  # idle until the next arrival
                    time.sleep(max(0.0, min(0.05, pending[k].arrival - (clock() - t0))))
                continue
            chosen = self._select()
            for mid in self.resident:
                want = mid in chosen
                if want != (mid in self.active):
                    self.batch.set_active(mid, want)
                    if want:
                        self.active.add(mid)
                    else:
                        self.active.discard(mid)
            self.batch.run(self.tick_iters)
            self.ticks += 1
            for mid in list(self.resident):
                if mid not in chosen:
                    continue
                req, nbytes = self.resident[mid]
                req.iterations += self.tick_iters
                if req.iterations >= self.iters:
                    Y, it = self.batch.get_Y(mid)
                    req.Y = Y
                    req.meta["device_iterations"] = it
                    req.finished = clock() - t0
                    self.batch.remove(mid)
                    del self.resident[mid]
                    self.active.discard(mid)
                    self.used -= nbytes
                    done.append(req)
        wall = clock() - t0
        return summarize(done, wall)

    def _select(self) -> set[int]:
        if self.policy == "all":
            return set(self.resident)

        def remaining(mid):
            req = self.resident[mid][0]
            return (self.iters - req.iterations) * float(req.n) ** 2

        chosen, pairs = set(), 0.0
        for mid in sorted(self.resident, key=lambda m: (remaining(m), m)):
            chosen.add(mid)
            pairs += 0.5 * float(self.resident[mid][0].n) ** 2
            if pairs >= self.fill_pairs:
                break
        return chosen

    def close(self):
        self.batch.close()


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


def serial_baseline(requests: list[Request], iters: int, config=None, clock=time.perf_counter) -> dict:
    """The same trace served one layout at a time (first come, first served)
    with the single-layout context API: the plain-run comparison point."""
    from . import Layout

    cfg = config if config is not None else tsgne_config_default()
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    lats = []
    for r in pending:
        now = clock() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        with Layout(cfg) as lay:
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

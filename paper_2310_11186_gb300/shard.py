"""One layout over several GPUs: the exact repulsion's tile-pair units divided
among the ranks of a torch.distributed group, one context per rank.

Every rank holds the whole layout, P and optimiser state (O(n + nnz)); only
the O(n^2) repulsion pass is divided.  Per iteration each rank

  1. enqueues its units [U r / w, U (r + 1) / w) of the U tile pairs
     (``tsgne_shard_repulsion``): forces into its int64 fixed-point
     accumulators, Z partials into its slots of the per-unit array;
  2. sums both arrays over the ranks in place (all-reduce; int64 and
     "x + 0" additions are exact, so the result does not depend on the
     reduction order);
  3. finishes the iteration (``tsgne_shard_step_finish``): Z in the fixed
     unit order, F^r, attraction and update of every row.

Every rank then holds the same bits as one context running ``tsgne_step``.
With the NCCL backend the all-reduce runs on the context's stream over the
library's device buffers (no copies); with gloo (CPU tests, or ranks that
share one GPU) the buffers go through host memory.  No kernel of one rank
ever waits on another rank: the only exchange is the host-issued
collective between two launches.
"""

from __future__ import annotations

from . import (DeviceArray, Layout, tsgne_shard_gradient_finish, tsgne_shard_repulsion, tsgne_shard_set,
               tsgne_shard_step_finish)


def unit_range(units: int, rank: int, world: int) -> tuple[int, int]:
    """Units [u0, u1) of rank ``rank`` out of ``world``: contiguous and as even
    as integer division allows (the library uses the same rule)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return units * rank // world, units * (rank + 1) // world


def tile_units(n: int, tile: int) -> int:
    """Tile pairs a <= b of a layout of n points in tiles of ``tile`` points."""
    nt = (n + tile - 1) // tile
    return nt * (nt + 1) // 2


def allreduce_sum_(tensors, group=None, stream=None):
    """Sums each tensor over the group's ranks in place.  NCCL: device
    tensors on ``stream``; any other backend: through host memory (the
    stream is synchronised first)."""
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)
    if backend == "nccl":
        with torch.cuda.stream(stream) if stream is not None else _null():
            for t in tensors:
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return
    if stream is not None:
        stream.synchronize()
    for t in tensors:
        h = t.cpu() if t.is_cuda else t
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        if t.is_cuda:
            t.copy_(h)  # on torch's current stream
    if stream is not None and any(t.is_cuda for t in tensors):
        stream.wait_stream(torch.cuda.current_stream())  # the finish call runs after the copies


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


class ShardedLayout:
    """A layout whose exact repulsion is divided over the ranks of ``group``
    (default: the default process group; rank and world from it).

    >>> lay = ShardedLayout(perplexity=30.0)   # after init_process_group
    >>> lay.build_P(row_ptr, col, X); lay.init_Y(Y0)
    >>> lay.run(1000); Y = lay.get_Y()          # same bits on every rank
    """

    def __init__(self, group=None, rank: int | None = None, world: int | None = None, **config):
        import torch.distributed as dist

        self.group = group
        if rank is None or world is None:
            rank = dist.get_rank(group)
            world = dist.get_world_size(group)
        self.rank, self.world = int(rank), int(world)
        self.layout = Layout(**config)
        self.exchanged_bytes = 0

    # ---- set-up (every rank passes the same inputs)
    def build_P(self, row_ptr, col, X):
        self.layout.build_P(row_ptr, col, X)
        tsgne_shard_set(self.layout.ctx, self.rank, self.world)

    def set_P(self, row_ptr, col, P):
        self.layout.set_P(row_ptr, col, P)
        tsgne_shard_set(self.layout.ctx, self.rank, self.world)

    def init_Y(self, Y0=None):
        self.layout.init_Y(Y0)

    # ---- one sharded pass
    def _pass(self):
        import torch

        U, u0, u1, acc, zunit = tsgne_shard_repulsion(self.layout.ctx)
        dev = torch.device("cuda", torch.cuda.current_device())
        a = torch.as_tensor(acc, device=dev)
        z = torch.as_tensor(zunit, device=dev)
        allreduce_sum_([a, z], group=self.group, stream=self.layout.stream)
        self.exchanged_bytes += a.numel() * 8 + z.numel() * 8
        return U, u0, u1

    def step(self):
        self._pass()
        tsgne_shard_step_finish(self.layout.ctx)

    def run(self, n_iter: int):
        for _ in range(int(n_iter)):
            self.step()
        self.layout.sync()

    def gradient(self, alpha: float = 1.0, out=None):
        """(g, Z) at the current layout from a sharded pass (no state change)."""
        self._pass()
        return tsgne_shard_gradient_finish(self.layout.ctx, alpha, out)

    # ---- local reads (every rank holds the whole state)
    def get_Y(self, out=None):
        return self.layout.get_Y(out)

    def kl(self):
        """KL of the current layout, its Z summed by this rank alone."""
        return self.layout.kl()

    def sync(self):
        self.layout.sync()

    def close(self):
        self.layout.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
        return False


__all__ = ["unit_range", "tile_units", "allreduce_sum_", "ShardedLayout", "DeviceArray"]

"""GB300-native t-SGNE layout loop: thin Python binding of libtsgne.so.

t-SGNE (Li, Xiao, Zhou, "Efficiently Visualizing Large Graphs", arXiv
2310.11186, Sec. 2.2) lays out the nodes of a graph G in 2-D by running t-SNE
(Sec. 2.1) with the neighbour graph taken from G.  All of the computation
runs in the CUDA kernels of ``libtsgne.so`` (declared in ``include/tsgne.h``);
this module only marshals arguments through ctypes.  The functions keep the
C names (``tsgne_build_P``, ``tsgne_step``, ``tsgne_run``, ``tsgne_kl``, ...);
``Layout`` wraps them in a small class.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA);
device tensors are passed to the library as device pointers.  There is no
CPU fallback: if the library is not built, every call raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "TsgneError",
    "Config",
    "lib",
    "library_path",
    "EXPORTS",
    "tsgne_config_default",
    "tsgne_create",
    "tsgne_destroy",
    "tsgne_last_error",
    "tsgne_status_string",
    "tsgne_build_P",
    "tsgne_set_P",
    "tsgne_get_sizes",
    "tsgne_get_P",
    "tsgne_init_Y",
    "tsgne_step",
    "tsgne_run",
    "tsgne_kl",
    "tsgne_gradient",
    "tsgne_get_Y",
    "tsgne_get_state",
    "tsgne_set_state",
    "tsgne_kernel_times",
    "tsgne_repulsion_shape",
    "tsgne_sync",
    "tsgne_repulsion_noalloc",
    "tsgne_shard_set",
    "tsgne_shard_repulsion",
    "tsgne_shard_step_finish",
    "tsgne_shard_gradient_finish",
    "tsgne_shortest_path_embedding",
    "tsgne_build_P_shortest_path",
    "NOALLOC_MAX_N",
    "DeviceArray",
    "Layout",
    "Batch",
    "ServerConfig",
    "Server",
    "server_estimate_bytes",
    "set_device_memory_limit",
    "device_memory_in_use",
    "KERNEL_CLASSES",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
# TSGNE_DEBUG=1 selects the index-checking debug build (build.build(debug=True))
library_path = os.path.join(_PKG, "lib", "libtsgne_debug.so" if os.environ.get("TSGNE_DEBUG") == "1"
                            else "libtsgne.so")

PTR_HOST, PTR_DEVICE = 0, 1
KERNEL_CLASSES = ("repulsion", "attract_update", "gradient", "kl", "build", "fix_forces", "attract_hubs",
                  "tree_build")

STATUS = {
    0: "TSGNE_OK",
    1: "TSGNE_ERR_INVALID_ARG",
    2: "TSGNE_ERR_BAD_CSR",
    3: "TSGNE_ERR_OOM",
    4: "TSGNE_ERR_CUDA",
    5: "TSGNE_ERR_NOT_BUILT",
    6: "TSGNE_ERR_NONFINITE",
    7: "TSGNE_ERR_TIMEOUT",
    8: "TSGNE_ERR_CANCELLED",
    9: "TSGNE_ERR_INDEX",
}


class TsgneError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


class Config(ctypes.Structure):
    """Mirror of ``tsgne_config``."""

    _fields_ = [
        ("perplexity", ctypes.c_float),
        ("k_nn", ctypes.c_int32),
        ("early_exag", ctypes.c_float),
        ("ee_iters", ctypes.c_int32),
        ("momentum0", ctypes.c_float),
        ("momentum1", ctypes.c_float),
        ("learning_rate", ctypes.c_float),
        ("min_gain", ctypes.c_float),
        ("bisect_tol", ctypes.c_float),
        ("bisect_max_iter", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("precision", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("spin_budget_cycles", ctypes.c_int64),
        ("repulsion", ctypes.c_int32),
        ("theta", ctypes.c_float),
        ("p_walks", ctypes.c_int32),
        ("p_walk_length", ctypes.c_int32),
    ]


_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_st = ctypes.c_int

# name -> (restype, argtypes); the declarations of include/tsgne.h
EXPORTS = {
    "tsgne_config_default": (None, [ctypes.POINTER(Config)]),
    "tsgne_create": (_st, [ctypes.POINTER(_p), ctypes.POINTER(Config), _p]),
    "tsgne_destroy": (None, [_p]),
    "tsgne_last_error": (ctypes.c_char_p, [_p]),
    "tsgne_status_string": (ctypes.c_char_p, [_st]),
    "tsgne_build_P": (_st, [_p, _i32, _p, _p, _p, _i32, _i32]),
    "tsgne_set_P": (_st, [_p, _i32, _p, _p, _p, _i32]),
    "tsgne_get_sizes": (_st, [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "tsgne_get_P": (_st, [_p, _p, _p, _p, _i32]),
    "tsgne_init_Y": (_st, [_p, _p, _i32]),
    "tsgne_step": (_st, [_p]),
    "tsgne_run": (_st, [_p, _i32]),
    "tsgne_kl": (_st, [_p, ctypes.POINTER(ctypes.c_double)]),
    "tsgne_gradient": (_st, [_p, ctypes.c_float, _p, ctypes.POINTER(ctypes.c_double), _i32]),
    "tsgne_get_Y": (_st, [_p, _p, _i32]),
    "tsgne_get_state": (_st, [_p, _p, _p, _p, ctypes.POINTER(_i32), _i32]),
    "tsgne_set_state": (_st, [_p, _p, _p, _p, _i32, _i32]),
    "tsgne_kernel_times": (_st, [_p, _p, _p, _i32, _i32]),
    "tsgne_repulsion_shape": (_st, [_p] + [ctypes.POINTER(_i32)] * 6),
    "tsgne_sync": (_st, [_p]),
    "tsgne_set_repulsion_shape": (_st, [_p, _i32, _i32, _i32]),
    "tsgne_autotune": (_st, [_p, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32), _p]),
    "tsgne_repulsion_noalloc": (_st, [_i32, _p, _p, _p, _p]),
    "tsgne_shard_set": (_st, [_p, _i32, _i32]),
    "tsgne_shard_repulsion": (_st, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                    ctypes.POINTER(_p), ctypes.POINTER(_i64), ctypes.POINTER(_p)]),
    "tsgne_shard_step_finish": (_st, [_p]),
    "tsgne_shard_gradient_finish": (_st, [_p, ctypes.c_float, _p, ctypes.POINTER(ctypes.c_double), _i32]),
    "tsgne_stream": (_st, [_p, ctypes.POINTER(_p)]),
    "tsgne_batch_create": (_st, [ctypes.POINTER(_p), ctypes.POINTER(Config), _i32, _p]),
    "tsgne_batch_destroy": (None, [_p]),
    "tsgne_batch_last_error": (ctypes.c_char_p, [_p]),
    "tsgne_batch_add": (_st, [_p, _i32, _p, _p, _p, _i32, _p, _i32, ctypes.POINTER(_i32)]),
    "tsgne_batch_add_ex": (_st, [_p, _i32, _p, _p, _p, _i32, _p, _i32, _i32, ctypes.POINTER(_i32)]),
    "tsgne_batch_prepare": (_st, [_p, _i32, _p, _p, _p, _i32, _p, _i32, _i32, _p, ctypes.POINTER(_p)]),
    "tsgne_batch_attach": (_st, [_p, _p, ctypes.POINTER(_i32)]),
    "tsgne_batch_discard": (None, [_p]),
    "tsgne_batch_remove": (_st, [_p, _i32]),
    "tsgne_batch_size": (_st, [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "tsgne_batch_run": (_st, [_p, _i32]),
    "tsgne_batch_get_Y": (_st, [_p, _i32, _p, ctypes.POINTER(_i32), _i32]),
    "tsgne_batch_set_tile": (_st, [_p, _i32]),
    "tsgne_batch_set_active": (_st, [_p, _i32, _i32]),
    "tsgne_batch_reset": (_st, [_p]),
    "tsgne_batch_autotune": (_st, [_p, _i32, ctypes.POINTER(_i32), _p]),
    "tsgne_batch_cached_tile": (_st, [_p, ctypes.POINTER(_i32)]),
    "tsgne_batch_set_shape": (_st, [_p, _i32, _i32]),
    "tsgne_batch_shape": (_st, [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "tsgne_batch_autotune_shapes": (_st, [_p, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _p]),
    "tsgne_shortest_path_embedding": (_st, [_i32, _p, _p, _p, _i32, _i32, _p, _i32, _p]),
    "tsgne_build_P_shortest_path": (_st, [_p, _i32, _p, _p, _p, _i32, _i32, _i32]),
    "tsgne_set_device_memory_limit": (None, [_i64]),
    "tsgne_device_memory_in_use": (_i64, []),
    "tsgne_server_config_default": (None, [_p]),
    "tsgne_server_estimate_bytes": (_i64, [_i32, _i64, _i32]),
    "tsgne_server_create": (_st, [ctypes.POINTER(_p), _p, _p, _p]),
    "tsgne_server_destroy": (None, [_p]),
    "tsgne_server_last_error": (ctypes.c_char_p, [_p]),
    "tsgne_server_submit": (_st, [_p, _i32, _p, _p, _p, _i32, _p, ctypes.POINTER(_i64)]),
    "tsgne_server_tick": (_st, [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "tsgne_server_finished": (_st, [_p, _p, _i32, ctypes.POINTER(_i32)]),
    "tsgne_server_status": (_st, [_p, _i64, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "tsgne_server_result": (_st, [_p, _i64, _p]),
    "tsgne_server_cancel": (_st, [_p, _i64]),
    "tsgne_server_usage": (_st, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
}

NOALLOC_MAX_N = 65536  # TSGNE_NOALLOC_MAX_N

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError(
                f"{library_path} is missing: build it with `python -m paper_2310_11186_gb300.build` "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(library_path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# ------------------------------------------------------------- marshalling

def _torch():
    try:
        import torch  # noqa: F401
        return torch
    except Exception:  # pragma: no cover
        return None


def _as_buffer(a, dtype):
    """(pointer, ptr_kind, keep-alive object) for a numpy array or torch tensor."""
    if a is None:
        return None, PTR_HOST, None
    torch = _torch()
    if torch is not None and isinstance(a, torch.Tensor):
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.int64: torch.int64}[np.dtype(dtype).type]
        t = a.contiguous()
        if t.dtype != tdt:
            t = t.to(tdt)
        kind = PTR_DEVICE if t.is_cuda else PTR_HOST
        return ctypes.c_void_p(t.data_ptr()), kind, t
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), PTR_HOST, arr


def _check(ctx, status):
    if status != 0:
        msg = lib().tsgne_last_error(ctx).decode() if ctx else ""
        raise TsgneError(status, msg)


# ------------------------------------------------------------ C functions

def tsgne_config_default(**overrides) -> Config:
    c = Config()
    lib().tsgne_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def tsgne_create(config: Config | None = None, stream=None):
    """Returns a context handle; stream is a torch.cuda.Stream, a raw handle or None."""
    handle = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
    st = lib().tsgne_create(ctypes.byref(handle), ctypes.byref(config) if config is not None else None, s)
    if st != 0:
        raise TsgneError(st, "tsgne_create failed")
    return handle


def tsgne_destroy(ctx) -> None:
    lib().tsgne_destroy(ctx)


def tsgne_last_error(ctx) -> str:
    return lib().tsgne_last_error(ctx).decode()


def tsgne_status_string(status: int) -> str:
    return lib().tsgne_status_string(status).decode()


def _same_kind(*bufs):
    kinds = {b[1] for b in bufs if b[0] is not None}
    if len(kinds) > 1:
        raise ValueError("inputs of one call must all be on the host or all on the device")
    return kinds.pop() if kinds else PTR_HOST


def tsgne_build_P(ctx, n, row_ptr, col_idx, X):
    _graph(int(n), row_ptr, col_idx)
    if len(X.shape) != 2 or int(X.shape[0]) != int(n):
        raise ValueError("X must be an n x d array")
    rp = _as_buffer(row_ptr, np.int64)
    ci = _as_buffer(col_idx, np.int32)
    x = _as_buffer(X, np.float32)
    d = int(X.shape[1])
    kind = _same_kind(rp, ci, x)
    _check(ctx, lib().tsgne_build_P(ctx, int(n), rp[0], ci[0], x[0], d, kind))


def tsgne_shortest_path_embedding(row_ptr, col_idx, targets, l0: int = 0, out=None, stream=None):
    """ShortestPath embedding (Sec. 2.3, Eq. 8): float32 n x d BFS distances to
    the targets, capped at l0 + 1 (l0 <= 0: floor(sqrt(|E|)))."""
    n = len(row_ptr) - 1
    _graph(n, row_ptr, col_idx)
    rp = _as_buffer(row_ptr, np.int64)
    ci = _as_buffer(col_idx, np.int32)
    tg = _as_buffer(targets, np.int32)
    kind = _same_kind(rp, ci, tg)
    d = len(targets)
    if out is None:
        if kind == PTR_DEVICE:
            torch = _torch()
            out = torch.empty((n, d), dtype=torch.float32, device=row_ptr.device)
        else:
            out = np.zeros((n, d), np.float32)
    if _numel(out) != n * d:
        raise ValueError(f"out must hold n x d = {n * d} float32 values, not {_numel(out)}")
    ob = _as_buffer(out, np.float32)
    if ob[1] != kind:
        raise ValueError("out must live where the inputs live")
    if ob[2] is not out and not (hasattr(out, "data_ptr") and ob[2].data_ptr() == out.data_ptr()):
        raise ValueError("out must be a contiguous float32 array")
    s = None if stream is None else ctypes.c_void_p(getattr(stream, "cuda_stream", stream))
    st = lib().tsgne_shortest_path_embedding(n, rp[0], ci[0], tg[0], d, int(l0), ob[0], kind, s)
    if st != 0:
        raise TsgneError(st, "tsgne_shortest_path_embedding failed")
    return out


def tsgne_build_P_shortest_path(ctx, n, row_ptr, col_idx, targets, l0: int = 0):
    _graph(int(n), row_ptr, col_idx)
    rp = _as_buffer(row_ptr, np.int64)
    ci = _as_buffer(col_idx, np.int32)
    tg = _as_buffer(targets, np.int32)
    kind = _same_kind(rp, ci, tg)
    _check(ctx, lib().tsgne_build_P_shortest_path(ctx, int(n), rp[0], ci[0], tg[0], len(targets), int(l0), kind))


def tsgne_set_P(ctx, n, row_ptr, col_idx, P):
    _graph(int(n), row_ptr, col_idx)
    if _numel(P) != _numel(col_idx):
        raise ValueError("P must hold one value per entry of col")
    rp = _as_buffer(row_ptr, np.int64)
    ci = _as_buffer(col_idx, np.int32)
    pv = _as_buffer(P, np.float32)
    kind = _same_kind(rp, ci, pv)
    _check(ctx, lib().tsgne_set_P(ctx, int(n), rp[0], ci[0], pv[0], kind))


def tsgne_get_sizes(ctx):
    n = _i32()
    nnz = _i64()
    _check(ctx, lib().tsgne_get_sizes(ctx, ctypes.byref(n), ctypes.byref(nnz)))
    return n.value, nnz.value


def tsgne_get_P(ctx):
    """(row_ptr int64[n+1], col int32[nnz], P float32[nnz]) as numpy arrays."""
    n, nnz = tsgne_get_sizes(ctx)
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1), np.float32)
    _check(ctx, lib().tsgne_get_P(ctx, rp.ctypes.data_as(_p), col.ctypes.data_as(_p), val.ctypes.data_as(_p),
                                  PTR_HOST))
    return rp, col[:nnz], val[:nnz]


def tsgne_init_Y(ctx, Y0=None):
    if Y0 is not None:
        _rows(Y0, tsgne_get_sizes(ctx)[0], 2, "Y0")
    y = _as_buffer(Y0, np.float32)
    _check(ctx, lib().tsgne_init_Y(ctx, y[0], y[1]))


def tsgne_step(ctx):
    _check(ctx, lib().tsgne_step(ctx))


def tsgne_run(ctx, n_iter: int):
    _check(ctx, lib().tsgne_run(ctx, int(n_iter)))


def tsgne_kl(ctx) -> float:
    v = ctypes.c_double()
    _check(ctx, lib().tsgne_kl(ctx, ctypes.byref(v)))
    return v.value


def _numel(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") else int(np.size(a))


def _out(n, out):
    if out is None:
        out = np.zeros((n, 2), np.float32)
    if _numel(out) != 2 * n:
        raise ValueError(f"output must hold n x 2 = {2 * n} float32 values, not {_numel(out)}")
    buf = _as_buffer(out, np.float32)
    if buf[2] is not out and not (hasattr(out, "data_ptr") and buf[2].data_ptr() == out.data_ptr()):
        raise ValueError("output must be a contiguous float32 array")
    return out, buf


def _rows(a, n: int, k: int, name: str):
    """Checks that an input holds n x k values (k = 0: n values) before the
    library reads it."""
    if a is None:
        return
    want = n * k if k else n
    if _numel(a) != want:
        raise ValueError(f"{name} must hold {want} values ({n} x {k or 1}), not {_numel(a)}")


def _graph(n: int, row_ptr, col):
    """row_ptr must hold n + 1 values and col at least row_ptr[n] (the
    library reads that many; it validates the values themselves)."""
    if n < 0 or _numel(row_ptr) != n + 1:
        raise ValueError("row_ptr must hold n + 1 values")
    m = int(row_ptr[-1]) if n >= 0 and _numel(row_ptr) > 0 else 0
    if m > 0 and (col is None or _numel(col) < m):
        raise ValueError(f"col must hold at least row_ptr[n] = {m} values")


def tsgne_gradient(ctx, alpha: float = 1.0, out=None):
    """(g n x 2, Z): gradient of Eq. 5 with P scaled by alpha, and the normaliser."""
    n, _ = tsgne_get_sizes(ctx)
    out, buf = _out(n, out)
    z = ctypes.c_double()
    _check(ctx, lib().tsgne_gradient(ctx, float(alpha), buf[0], ctypes.byref(z), buf[1]))
    return out, z.value


def tsgne_shard_set(ctx, rank: int, world: int):
    _check(ctx, lib().tsgne_shard_set(ctx, int(rank), int(world)))


class DeviceArray:
    """A borrowed device buffer of the library (pointer, length, dtype),
    exposed through __cuda_array_interface__ so torch can wrap it in place
    (torch.as_tensor(arr, device=...)) without a copy."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.ptr, self.count, self.typestr = int(ptr), int(count), typestr

    @property
    def __cuda_array_interface__(self):
        return {"shape": (self.count,), "typestr": self.typestr, "data": (self.ptr, False), "version": 3,
                "strides": None, "stream": None}


def tsgne_shard_repulsion(ctx):
    """Enqueues this context's share of the exact repulsion pass; returns
    (units, u0, u1, acc, zunit): acc (int64, 2 n) and zunit (float64, units)
    are the context's device buffers to be summed over all shares in place."""
    U = _i64()
    u0 = _i32()
    u1 = _i32()
    acc = _p()
    cnt = _i64()
    z = _p()
    _check(ctx, lib().tsgne_shard_repulsion(ctx, ctypes.byref(U), ctypes.byref(u0), ctypes.byref(u1),
                                            ctypes.byref(acc), ctypes.byref(cnt), ctypes.byref(z)))
    return (U.value, u0.value, u1.value, DeviceArray(acc.value, cnt.value, "<i8"),
            DeviceArray(z.value, U.value, "<f8"))


def tsgne_shard_step_finish(ctx):
    _check(ctx, lib().tsgne_shard_step_finish(ctx))


def tsgne_shard_gradient_finish(ctx, alpha: float = 1.0, out=None):
    n, _ = tsgne_get_sizes(ctx)
    out, buf = _out(n, out)
    z = ctypes.c_double()
    _check(ctx, lib().tsgne_shard_gradient_finish(ctx, float(alpha), buf[0], ctypes.byref(z), buf[1]))
    return out, z.value


def tsgne_get_Y(ctx, out=None):
    n, _ = tsgne_get_sizes(ctx)
    out, buf = _out(n, out)
    _check(ctx, lib().tsgne_get_Y(ctx, buf[0], buf[1]))
    return out


def tsgne_get_state(ctx):
    n, _ = tsgne_get_sizes(ctx)
    Y = np.zeros((n, 2), np.float32)
    U = np.zeros((n, 2), np.float32)
    G = np.zeros((n, 2), np.float32)
    it = _i32()
    _check(ctx, lib().tsgne_get_state(ctx, Y.ctypes.data_as(_p), U.ctypes.data_as(_p), G.ctypes.data_as(_p),
                                      ctypes.byref(it), PTR_HOST))
    return Y, U, G, it.value


def tsgne_set_state(ctx, Y, update=None, gains=None, iteration=0):
    n = tsgne_get_sizes(ctx)[0]
    _rows(Y, n, 2, "Y")
    _rows(update, n, 2, "update")
    _rows(gains, n, 2, "gains")
    y = _as_buffer(Y, np.float32)
    u = _as_buffer(update, np.float32)
    g = _as_buffer(gains, np.float32)
    kind = _same_kind(y, u, g)
    _check(ctx, lib().tsgne_set_state(ctx, y[0], u[0], g[0], int(iteration), kind))


def tsgne_kernel_times(ctx, reset: bool = False):
    """{class: (ms, launches)} accumulated in profile mode."""
    ms = np.zeros(len(KERNEL_CLASSES))
    nl = np.zeros(len(KERNEL_CLASSES), np.int64)
    _check(ctx, lib().tsgne_kernel_times(ctx, ms.ctypes.data_as(_p), nl.ctypes.data_as(_p), len(KERNEL_CLASSES),
                                         int(bool(reset))))
    return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(KERNEL_CLASSES)}


def tsgne_repulsion_shape(ctx):
    vals = [_i32() for _ in range(6)]
    _check(ctx, lib().tsgne_repulsion_shape(ctx, *[ctypes.byref(v) for v in vals]))
    keys = ("grid", "block", "i_per_thread", "j_tile", "j_chunks", "n_pad")
    return {k: v.value for k, v in zip(keys, vals)}


def tsgne_sync(ctx):
    _check(ctx, lib().tsgne_sync(ctx))


def tsgne_repulsion_noalloc(Y, frep_out=None, z_out=None, stream=None):
    """Repulsion pass without any device allocation by the library.

    For callers that cannot allocate device memory (a host framework owns the
    memory budget, or allocation would synchronise the device): Y, frep_out
    (n x 2 float32) and z_out (1 float64) are CUDA tensors owned by the caller;
    temporaries live in a static device array of the library.  Returns
    (frep_out, z_out) with F^r_i = sum_{j != i} w_ij^2 (y_i - y_j) and
    Z = sum_{k != l} w_kl.  At most NOALLOC_MAX_N points.  Calls that overlap
    on the GPU share that array and race: keep them on one stream.
    """
    torch = _torch()
    if torch is None or not isinstance(Y, torch.Tensor) or not Y.is_cuda:
        raise ValueError("Y must be a CUDA tensor")
    if Y.dim() != 2 or Y.shape[1] != 2:
        raise ValueError(f"Y must have shape (n, 2), got {tuple(Y.shape)}")
    Yc = Y.contiguous().float()
    n = int(Yc.shape[0])
    if frep_out is None:
        frep_out = torch.empty((n, 2), dtype=torch.float32, device=Yc.device)
    if z_out is None:
        z_out = torch.empty((1,), dtype=torch.float64, device=Yc.device)
    if not (frep_out.is_cuda and frep_out.dtype == torch.float32 and frep_out.is_contiguous()):
        raise ValueError("frep_out must be a contiguous float32 CUDA tensor")
    if tuple(frep_out.shape) != (n, 2):
        raise ValueError(f"frep_out must have shape ({n}, 2), got {tuple(frep_out.shape)}")
    if not (z_out.is_cuda and z_out.dtype == torch.float64) or z_out.numel() < 1:
        raise ValueError("z_out must be a float64 CUDA tensor with at least one element")
    if frep_out.device != Yc.device or z_out.device != Yc.device:
        raise ValueError("Y, frep_out and z_out must be on the same device")
    with torch.cuda.device(Yc.device):
        s = stream if stream is not None else torch.cuda.current_stream(Yc.device)
        handle = ctypes.c_void_p(getattr(s, "cuda_stream", s))
        st = lib().tsgne_repulsion_noalloc(n, ctypes.c_void_p(Yc.data_ptr()), ctypes.c_void_p(frep_out.data_ptr()),
                                           ctypes.c_void_p(z_out.data_ptr()), handle)
    if st != 0:
        raise TsgneError(st, lib().tsgne_last_error(None).decode() or "tsgne_repulsion_noalloc failed")
    return frep_out, z_out


# ------------------------------------------------------------ convenience

class Layout:
    """One graph's layout state on the GPU.

    >>> lay = Layout(perplexity=30.0)
    >>> lay.build_P(row_ptr, col, X)      # CSR + embedding (host or device)
    >>> lay.init_Y(Y0)                    # or None: N(0, 1e-4^2) from the seed
    >>> lay.run(1000); Y = lay.get_Y(); kl = lay.kl()
    """

    def __init__(self, config: Config | None = None, stream=None, **overrides):
        cfg = config if config is not None else tsgne_config_default()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.config = cfg
        self._stream = stream
        if stream is None:
            torch = _torch()
            if torch is not None and torch.cuda.is_available():
                self._stream = torch.cuda.Stream()
        self.ctx = tsgne_create(cfg, self._stream)

    @property
    def stream(self):
        return self._stream

    def _order_after_torch(self):
        torch = _torch()
        if torch is not None and self._stream is not None and hasattr(self._stream, "wait_stream"):
            self._stream.wait_stream(torch.cuda.current_stream())

    def build_P(self, row_ptr, col, X):
        self._order_after_torch()
        tsgne_build_P(self.ctx, len(row_ptr) - 1, row_ptr, col, X)

    def build_P_shortest_path(self, row_ptr, col, targets, l0: int = 0):
        """The paper's pipeline: ShortestPath embedding (Eq. 8) then P."""
        self._order_after_torch()
        tsgne_build_P_shortest_path(self.ctx, len(row_ptr) - 1, row_ptr, col, targets, l0)

    def set_P(self, row_ptr, col, P):
        self._order_after_torch()
        tsgne_set_P(self.ctx, len(row_ptr) - 1, row_ptr, col, P)

    def init_Y(self, Y0=None):
        self._order_after_torch()
        tsgne_init_Y(self.ctx, Y0)

    def step(self):
        tsgne_step(self.ctx)

    def run(self, n_iter):
        tsgne_run(self.ctx, n_iter)

    def kl(self):
        return tsgne_kl(self.ctx)

    def gradient(self, alpha=1.0, out=None):
        return tsgne_gradient(self.ctx, alpha, out)

    REPULSION_SHAPES = ((2, 16, 1), (1, 16, 1), (2, 8, 1), (1, 8, 1), (0, 0, 0))

    def set_repulsion_shape(self, tile_warps: int, i_per_lane: int, symmetric: bool = True):
        _check(self.ctx, lib().tsgne_set_repulsion_shape(self.ctx, int(tile_warps), int(i_per_lane),
                                                         1 if symmetric else 0))

    def autotune(self, trial_passes: int = 3):
        """Times each shape of the exact pass; keeps the fastest.  Returns
        ((warps, i-points per lane, symmetric), {shape name: ms per pass})."""
        w, ri, sym = _i32(), _i32(), _i32()
        ms = np.zeros(5, np.float32)
        _check(self.ctx, lib().tsgne_autotune(self.ctx, int(trial_passes), ctypes.byref(w), ctypes.byref(ri),
                                              ctypes.byref(sym), ms.ctypes.data_as(_p)))
        names = [f"sym_{a}x{b}" if c else "ordered" for a, b, c in self.REPULSION_SHAPES]
        return (w.value, ri.value, sym.value), {k: float(v) for k, v in zip(names, ms)}

    def get_Y(self, out=None):
        return tsgne_get_Y(self.ctx, out)

    def get_P(self):
        return tsgne_get_P(self.ctx)

    def get_state(self):
        return tsgne_get_state(self.ctx)

    def set_state(self, Y, update=None, gains=None, iteration=0):
        self._order_after_torch()
        tsgne_set_state(self.ctx, Y, update, gains, iteration)

    def sizes(self):
        return tsgne_get_sizes(self.ctx)

    def kernel_times(self, reset=False):
        return tsgne_kernel_times(self.ctx, reset)

    def repulsion_shape(self):
        return tsgne_repulsion_shape(self.ctx)

    def sync(self):
        tsgne_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            tsgne_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches

class Batch:
    """Many layouts advanced together (the ``tsgne_batch_*`` C calls).

    >>> b = Batch(tile_warps=2)
    >>> ids = [b.add(g.row_ptr, g.col, X, Y0) for g, X, Y0 in graphs]
    >>> b.run(100); Y, it = b.get_Y(ids[0])
    """

    def __init__(self, config: Config | None = None, tile_warps: int = 0, stream=None, **overrides):
        cfg = config if config is not None else tsgne_config_default()
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.config = cfg
        self._stream = stream
        if stream is None:
            torch = _torch()
            if torch is not None and torch.cuda.is_available():
                self._stream = torch.cuda.Stream()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(getattr(self._stream, "cuda_stream", self._stream)) if self._stream is not None else None
        st = lib().tsgne_batch_create(ctypes.byref(h), ctypes.byref(cfg), int(tile_warps), s)
        if st != 0:
            raise TsgneError(st, "tsgne_batch_create failed")
        self.h = h
        self.sizes = {}

    def _check(self, st):
        if st != 0:
            raise TsgneError(st, lib().tsgne_batch_last_error(self.h).decode())

    def add(self, row_ptr, col, X, Y0=None, repulsion=None) -> int:
        """Adds a member; repulsion 0 (exact) or 1 (tree code), default the
        batch configuration's."""
        n = len(row_ptr) - 1
        _graph(n, row_ptr, col)
        if len(X.shape) != 2 or int(X.shape[0]) != n:
            raise ValueError("X must be an n x d array")
        _rows(Y0, n, 2, "Y0")
        rp = _as_buffer(row_ptr, np.int64)
        ci = _as_buffer(col, np.int32)
        x = _as_buffer(X, np.float32)
        y = _as_buffer(Y0, np.float32)
        kind = _same_kind(rp, ci, x, y)
        out = _i32()
        n = len(row_ptr) - 1
        if repulsion is None:
            self._check(lib().tsgne_batch_add(self.h, n, rp[0], ci[0], x[0], int(X.shape[1]), y[0], kind,
                                              ctypes.byref(out)))
        else:
            self._check(lib().tsgne_batch_add_ex(self.h, n, rp[0], ci[0], x[0], int(X.shape[1]), y[0], kind,
                                                 int(repulsion), ctypes.byref(out)))
        self.sizes[out.value] = n
        return out.value

    def remove(self, mid: int):
        self._check(lib().tsgne_batch_remove(self.h, int(mid)))
        self.sizes.pop(mid, None)

    def size(self):
        m, w, u = _i32(), _i32(), _i64()
        self._check(lib().tsgne_batch_size(self.h, ctypes.byref(m), ctypes.byref(w), ctypes.byref(u)))
        return {"members": m.value, "tile_warps": w.value, "units": u.value}

    def run(self, n_iter: int):
        self._check(lib().tsgne_batch_run(self.h, int(n_iter)))

    def get_Y(self, mid: int, out=None):
        if mid not in self.sizes:
            raise TsgneError(1, f"unknown member id {mid}")
        n = self.sizes[mid]
        out, buf = _out(n, out)
        it = _i32()
        self._check(lib().tsgne_batch_get_Y(self.h, int(mid), buf[0], ctypes.byref(it), buf[1]))
        return out, it.value

    def set_active(self, mid: int, active: bool = True):
        """Inactive members keep their state and are skipped by run()."""
        self._check(lib().tsgne_batch_set_active(self.h, int(mid), int(bool(active))))

    def set_tile(self, tile_warps: int):
        self._check(lib().tsgne_batch_set_tile(self.h, int(tile_warps)))

    def reset(self):
        self._check(lib().tsgne_batch_reset(self.h))

    BATCH_SHAPES = ((1, 16), (2, 16), (4, 16), (1, 8), (2, 8), (4, 8))

    def autotune(self, trial_iters: int = 3):
        """Tile warps only (16 i-points per lane): (chosen warps, {warps: ms})."""
        chosen = _i32()
        ms = np.zeros(3, np.float32)
        self._check(lib().tsgne_batch_autotune(self.h, int(trial_iters), ctypes.byref(chosen),
                                               ms.ctypes.data_as(_p)))
        return chosen.value, dict(zip((1, 2, 4), ms.tolist()))

    def autotune_shapes(self, trial_iters: int = 3):
        """Every compiled shape: ((warps, i-points per lane), {"WxRI": ms})."""
        w, ri = _i32(), _i32()
        ms = np.zeros(6, np.float32)
        self._check(lib().tsgne_batch_autotune_shapes(self.h, int(trial_iters), ctypes.byref(w), ctypes.byref(ri),
                                                      ms.ctypes.data_as(_p)))
        return (w.value, ri.value), {f"{a}x{b}": float(t) for (a, b), t in zip(self.BATCH_SHAPES, ms)}

    def set_shape(self, tile_warps: int, i_per_lane: int):
        self._check(lib().tsgne_batch_set_shape(self.h, int(tile_warps), int(i_per_lane)))

    def shape(self):
        w, ri = _i32(), _i32()
        self._check(lib().tsgne_batch_shape(self.h, ctypes.byref(w), ctypes.byref(ri)))
        return w.value, ri.value

    def cached_tile(self) -> int:
        w = _i32()
        self._check(lib().tsgne_batch_cached_tile(self.h, ctypes.byref(w)))
        return w.value

    def close(self):
        if getattr(self, "h", None):
            lib().tsgne_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving

class ServerConfig(ctypes.Structure):
    """Mirror of ``tsgne_server_config``."""

    _fields_ = [
        ("budget_bytes", ctypes.c_int64),
        ("iters", ctypes.c_int32),
        ("tick_iters", ctypes.c_int32),
        ("max_members", ctypes.c_int32),
        ("tile_warps", ctypes.c_int32),
        ("policy", ctypes.c_int32),
        ("aging_ticks", ctypes.c_int32),
        ("fill_pairs", ctypes.c_double),
        ("tree_min_n", ctypes.c_int32),
    ]


def set_device_memory_limit(nbytes: int):
    """tsgne_set_device_memory_limit: cap on the library's device bytes (<= 0: none)."""
    lib().tsgne_set_device_memory_limit(int(nbytes))


def device_memory_in_use() -> int:
    """tsgne_device_memory_in_use."""
    return int(lib().tsgne_device_memory_in_use())


def server_estimate_bytes(n: int, nnz: int, tile_warps: int) -> int:
    """tsgne_server_estimate_bytes (host arithmetic; no GPU needed)."""
    return int(lib().tsgne_server_estimate_bytes(int(n), int(nnz), int(tile_warps)))


class Server:
    """The ``tsgne_server_*`` C calls: queue, admission by device-memory
    budget, shortest-remaining-work scheduling and retirement all run in the
    library; this class only marshals.

    >>> srv = Server(iters=500)
    >>> rid = srv.submit(g.row_ptr, g.col, X)
    >>> while srv.tick()[0] or srv.tick()[1]: ...
    >>> Y = srv.result(rid)
    """

    STATES = ("queued", "resident", "done", "cancelled")

    def __init__(self, config: Config | None = None, stream=None, **server_fields):
        sc = ServerConfig()
        lib().tsgne_server_config_default(ctypes.byref(sc))
        for k, v in server_fields.items():
            setattr(sc, k, v)
        self.server_config = sc
        self.config = config if config is not None else tsgne_config_default()
        self._stream = stream
        if stream is None:
            torch = _torch()
            if torch is not None and torch.cuda.is_available():
                self._stream = torch.cuda.Stream()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(getattr(self._stream, "cuda_stream", self._stream)) if self._stream is not None else None
        st = lib().tsgne_server_create(ctypes.byref(h), ctypes.byref(sc), ctypes.byref(self.config), s)
        if st != 0:
            raise TsgneError(st, "tsgne_server_create failed")
        self.h = h
        self.sizes = {}

    def _check(self, st):
        if st != 0:
            raise TsgneError(st, lib().tsgne_server_last_error(self.h).decode())

    def submit(self, row_ptr, col, X, Y0=None) -> int:
        rp = np.ascontiguousarray(row_ptr, np.int64)
        ci = np.ascontiguousarray(col, np.int32)
        x = np.ascontiguousarray(X, np.float32)
        y = None if Y0 is None else np.ascontiguousarray(Y0, np.float32)
        rid = _i64()
        n = rp.size - 1
        _graph(n, rp, ci)
        if x.ndim != 2 or x.shape[0] != n:
            raise ValueError("X must be an n x d array")
        _rows(y, n, 2, "Y0")
        self._check(lib().tsgne_server_submit(self.h, n, rp.ctypes.data_as(_p), ci.ctypes.data_as(_p) if ci.size else None,
                                              x.ctypes.data_as(_p), int(x.shape[1]),
                                              None if y is None else y.ctypes.data_as(_p), ctypes.byref(rid)))
        self.sizes[rid.value] = n
        return rid.value

    def tick(self):
        """One scheduling round; returns (resident, queued, retired)."""
        r, q, d = _i32(), _i32(), _i32()
        self._check(lib().tsgne_server_tick(self.h, ctypes.byref(r), ctypes.byref(q), ctypes.byref(d)))
        return r.value, q.value, d.value

    def finished(self, capacity: int = 1024):
        ids = np.zeros(max(1, capacity), np.int64)
        k = _i32()
        self._check(lib().tsgne_server_finished(self.h, ids.ctypes.data_as(_p), int(capacity), ctypes.byref(k)))
        return ids[: k.value].tolist()

    def status(self, rid: int):
        st, it = _i32(), _i32()
        self._check(lib().tsgne_server_status(self.h, int(rid), ctypes.byref(st), ctypes.byref(it)))
        return self.STATES[st.value], it.value

    def result(self, rid: int):
        out = np.empty((self.sizes[rid], 2), np.float32)
        self._check(lib().tsgne_server_result(self.h, int(rid), out.ctypes.data_as(_p)))
        self.sizes.pop(rid, None)
        return out

    def cancel(self, rid: int):
        self._check(lib().tsgne_server_cancel(self.h, int(rid)))

    def usage(self):
        u, r, q = _i64(), _i32(), _i32()
        self._check(lib().tsgne_server_usage(self.h, ctypes.byref(u), ctypes.byref(r), ctypes.byref(q)))
        return {"used_bytes": u.value, "resident": r.value, "queued": q.value}

    def close(self):
        if getattr(self, "h", None):
            lib().tsgne_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

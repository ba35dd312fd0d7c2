"""FP64 CPU oracle for the t-SGNE layout loop (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product (the CUDA library and its Python
binding) never does, and this package never imports the product.

The arithmetic lives in ``tsgne_oracle.c`` (plain C, double precision, one
function per definition of the paper, each citing its section / equation).
This module compiles it with gcc and marshals numpy arrays; it adds no
arithmetic of its own except where noted (the learning-rate rule and the
thread split of the quadratic row sums).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle.py`` (closed forms, brute force, finite differences and
invariants).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsgne_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libtsgne_oracle.so")
_lib = None
_lock = threading.Lock()

_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (IEEE semantics, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.tsgo_check_csr.argtypes = [_i32, _p, _p]
            lib.tsgo_check_csr.restype = ctypes.c_int
            lib.tsgo_structure.argtypes = [_i32, _p, _p, _p, _p]
            lib.tsgo_structure.restype = _i64
            lib.tsgo_transpose_slots.argtypes = [_i32, _p, _p, _p]
            lib.tsgo_transpose_slots.restype = ctypes.c_int
            lib.tsgo_cond_affinity.argtypes = [_i32, _p, _p, _p, _i32, _dbl, _dbl, _i32, _p, _p, _p]
            lib.tsgo_cond_affinity.restype = ctypes.c_int
            lib.tsgo_joint_P.argtypes = [_i32, _p, _p, _p, _p, _p]
            lib.tsgo_joint_P.restype = ctypes.c_int
            lib.tsgo_Z.argtypes = [_i32, _p]
            lib.tsgo_Z.restype = _dbl
            lib.tsgo_kl.argtypes = [_i32, _p, _p, _p, _p, _p]
            lib.tsgo_kl.restype = _dbl
            lib.tsgo_gradient.argtypes = [_i32, _p, _p, _p, _p, _dbl, _p, _p]
            lib.tsgo_gradient.restype = ctypes.c_int
            lib.tsgo_repulsion_rows.argtypes = [_i32, _p, _i32, _i32, _p, _p]
            lib.tsgo_repulsion_rows.restype = ctypes.c_int
            lib.tsgo_attraction_rows.argtypes = [_i32, _p, _p, _p, _p, _p, _i32, _p]
            lib.tsgo_attraction_rows.restype = ctypes.c_int
            lib.tsgo_optimize.argtypes = [_i32, _p, _p, _p, _p, _p, _p, _i32, _i32, _dbl, _i32, _dbl, _dbl, _dbl, _dbl]
            lib.tsgo_optimize.restype = ctypes.c_int
            lib.tsgo_shortest_path.argtypes = [_i32, _p, _p, _p, _i32, _i32, _p]
            lib.tsgo_shortest_path.restype = ctypes.c_int
            lib.tsgo_bfs_knn.argtypes = [_i32, _p, _p, _i32, _p, _p]
            lib.tsgo_bfs_knn.restype = ctypes.c_int
            lib.tsgo_repulsion_tree.argtypes = [_i32, _p, _dbl, _i32, _p, _p, _p]
            lib.tsgo_repulsion_tree.restype = ctypes.c_int
            lib.tsgo_repulsion_tree_bounds.argtypes = [_i32, _p, _dbl, _i32, _p, _p, _p, _p]
            lib.tsgo_repulsion_tree_bounds.restype = ctypes.c_int
            lib.tsgo_tree_mutation.argtypes = [_i32]
            lib.tsgo_tree_mutation.restype = None
            lib.tsgo_gradient_tree.argtypes = [_i32, _p, _p, _p, _p, _dbl, _dbl, _i32, _p, _p]
            lib.tsgo_gradient_tree.restype = ctypes.c_int
            lib.tsgo_random_walk_counts.argtypes = [_i32, _p, _p, _p, _i32, _i32, _i32, ctypes.c_uint64, _p, _p, _p]
            lib.tsgo_random_walk_counts.restype = ctypes.c_int
            lib.tsgo_random_walk_pcond.argtypes = [_i32, _p, _p, _p, _i32, _p, _p, _p]
            lib.tsgo_random_walk_pcond.restype = ctypes.c_int
            lib.tsgo_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.tsgo_splitmix64.restype = ctypes.c_uint64
            lib.tsgo_gradient_rows.argtypes = [_i32, _p, _p, _p, _p, _dbl, _dbl, _p, _i32, _p]
            lib.tsgo_gradient_rows.restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(st: int, what: str):
    if st < 0:
        raise OracleError(f"{what}: status {st}")


def check_csr(n, row_ptr, col) -> int:
    rp, c = _c(row_ptr, np.int64), _c(col, np.int32)
    if rp.size != n + 1:
        return -1
    return _load().tsgo_check_csr(n, _ptr(rp), _ptr(c if c.size else np.zeros(1, np.int32)))


def structure(n, row_ptr, col):
    """Symmetric, sorted, unique, loop-free neighbour structure (Eq. 7)."""
    rp, c = _c(row_ptr, np.int64), _c(col, np.int32)
    if rp.size != n + 1:
        raise OracleError("row_ptr size")
    out_rp = np.zeros(n + 1, np.int64)
    out_col = np.zeros(max(1, 2 * int(rp[-1])), np.int32)
    nnz = _load().tsgo_structure(n, _ptr(rp), _ptr(c if c.size else np.zeros(1, np.int32)), _ptr(out_rp), _ptr(out_col))
    _check(nnz, "structure")
    return out_rp, out_col[:nnz].copy()


def transpose_slots(n, rp, col):
    rp, col = _c(rp, np.int64), _c(col, np.int32)
    t = np.zeros(max(1, col.size), np.int64)
    _check(_load().tsgo_transpose_slots(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)), _ptr(t)), "tslot")
    return t[: col.size]


def cond_affinity(n, rp, col, X, perplexity, tol=1e-5, max_iter=100):
    """p_{j|i} over N(i) (Eq. 2) with the Sec. 2.1 bisection; returns (pcond, beta, iters)."""
    rp, col = _c(rp, np.int64), _c(col, np.int32)
    Xd = _c(X, np.float64)
    d = Xd.shape[1]
    pc = np.zeros(max(1, col.size))
    beta = np.zeros(max(1, n))
    iters = np.zeros(max(1, n), np.int32)
    st = _load().tsgo_cond_affinity(
        n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)), _ptr(Xd), d, float(perplexity),
        float(tol), int(max_iter), _ptr(pc), _ptr(beta), _ptr(iters))
    _check(st, "cond_affinity")
    return pc[: col.size], beta[:n], iters[:n]


def joint_P(n, rp, col, pcond):
    """p_ij of Eq. 3 normalised to sum 1; returns (P, T)."""
    rp, col, pc = _c(rp, np.int64), _c(col, np.int32), _c(pcond, np.float64)
    P = np.zeros(max(1, col.size))
    T = ctypes.c_double(0.0)
    st = _load().tsgo_joint_P(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)),
                              _ptr(pc if pc.size else np.zeros(1)), _ptr(P), ctypes.byref(T))
    _check(st, "joint_P")
    return P[: col.size], T.value


def build_P(n, row_ptr, col, X, perplexity, tol=1e-5, max_iter=100):
    """Structure + conditional + joint affinities: returns (rp, col, P)."""
    rp, c = structure(n, row_ptr, col)
    pc, _, _ = cond_affinity(n, rp, c, X, perplexity, tol, max_iter)
    P, _ = joint_P(n, rp, c, pc)
    return rp, c, P


def Z(Y) -> float:
    Yd = _c(Y, np.float64)
    return _load().tsgo_Z(Yd.shape[0], _ptr(Yd))


def kl(n, rp, col, P, Y):
    """Eq. 5 objective; returns (KL, Z)."""
    rp, col, P, Yd = _c(rp, np.int64), _c(col, np.int32), _c(P, np.float64), _c(Y, np.float64)
    z = ctypes.c_double(0.0)
    v = _load().tsgo_kl(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)),
                        _ptr(P if P.size else np.zeros(1)), _ptr(Yd), ctypes.byref(z))
    return v, z.value


def gradient(n, rp, col, P, Y, alpha=1.0):
    """Gradient of Eq. 5 with exaggeration alpha; returns (G n x 2, Z)."""
    rp, col, P, Yd = _c(rp, np.int64), _c(col, np.int32), _c(P, np.float64), _c(Y, np.float64)
    G = np.zeros((n, 2))
    z = ctypes.c_double(0.0)
    st = _load().tsgo_gradient(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)),
                               _ptr(P if P.size else np.zeros(1)), _ptr(Yd), float(alpha), _ptr(G), ctypes.byref(z))
    _check(st, "gradient")
    return G, z.value


def repulsion_rows(Y, i0, i1):
    """(F_rep rows i0..i1-1, zrow) with zrow_i = sum_{j != i} w_ij."""
    Yd = _c(Y, np.float64)
    n = Yd.shape[0]
    F = np.zeros((max(1, i1 - i0), 2))
    zr = np.zeros(max(1, i1 - i0))
    _check(_load().tsgo_repulsion_rows(n, _ptr(Yd), i0, i1, _ptr(F), _ptr(zr)), "repulsion_rows")
    return F[: i1 - i0], zr[: i1 - i0]


def repulsion_tree(Y, theta, bucket=4):
    """Tree-code approximation of the repulsive sums (steps in the C source):
    returns (F_rep n x 2, zrow n, Z) in the input order.  theta = 0 gives the
    exact sums of repulsion_rows."""
    Yd = _c(Y, np.float64)
    n = Yd.shape[0]
    F = np.zeros((n, 2))
    zr = np.zeros(n)
    z = ctypes.c_double(0.0)
    _check(_load().tsgo_repulsion_tree(n, _ptr(Yd), float(theta), int(bucket), _ptr(F), _ptr(zr), ctypes.byref(z)),
           "repulsion_tree")
    return F, zr, z.value


def repulsion_tree_bounds(Y, theta, bucket=4):
    """repulsion_tree plus per-row error bounds against the exact sums:
    returns (F_rep, zrow, Z, bZ, bF) where bZ and bF are n x 2 arrays
    (centre-rounding part, second-order remainder part) bounding
    |zrow_i - exact zrow_i| and the Euclidean |F_i - exact F_i|."""
    Yd = _c(Y, np.float64)
    n = Yd.shape[0]
    F = np.zeros((n, 2))
    zr = np.zeros(n)
    b = np.zeros((n, 4))
    z = ctypes.c_double(0.0)
    _check(_load().tsgo_repulsion_tree_bounds(n, _ptr(Yd), float(theta), int(bucket), _ptr(F), _ptr(zr),
                                              ctypes.byref(z), _ptr(b)), "repulsion_tree_bounds")
    return F, zr, z.value, b[:, 0:2].copy(), b[:, 2:4].copy()


def tree_mutation(which: int) -> None:
    """Plants one of the tree code's numbered mistakes (0 = none); for the
    tests that show the bound check catches them."""
    _load().tsgo_tree_mutation(int(which))


def gradient_tree(n, rp, col, P, Y, alpha=1.0, theta=0.5, bucket=4):
    """Gradient of Eq. 5 with the tree code's repulsive sums and Z; returns (G, Z)."""
    rp, col, P, Yd = _c(rp, np.int64), _c(col, np.int32), _c(P, np.float64), _c(Y, np.float64)
    G = np.zeros((n, 2))
    z = ctypes.c_double(0.0)
    st = _load().tsgo_gradient_tree(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)),
                                    _ptr(P if P.size else np.zeros(1)), _ptr(Yd), float(alpha), float(theta),
                                    int(bucket), _ptr(G), ctypes.byref(z))
    _check(st, "gradient_tree")
    return G, z.value


def gradient_rows(n, rp, col, P, Y, alpha, Z, rows):
    """Gradient rows (Eq. 5 derivative) for a given Z; returns len(rows) x 2."""
    rp, col, P, Yd = _c(rp, np.int64), _c(col, np.int32), _c(P, np.float64), _c(Y, np.float64)
    rows = _c(rows, np.int32)
    G = np.zeros((max(1, rows.size), 2))
    st = _load().tsgo_gradient_rows(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)),
                                    _ptr(P if P.size else np.zeros(1)), _ptr(Yd), float(alpha), float(Z), _ptr(rows),
                                    rows.size, _ptr(G))
    _check(st, "gradient_rows")
    return G[: rows.size]


def splitmix64(seed: int, k: int) -> int:
    """Output number k >= 1 of the SplitMix64 sequence seeded with seed."""
    return int(_load().tsgo_splitmix64(seed & (2 ** 64 - 1), k))


def random_walk_counts(n, rp, col, X, walks, length, seed=0):
    """Eq. 6 walk counts: (wrp, wcol, wcnt), per node the distinct end points
    j != i of its walks (increasing) and how many walks ended there."""
    rp, col, Xd = _c(rp, np.int64), _c(col, np.int32), _c(X, np.float64)
    d = Xd.shape[1]
    cap = max(1, n * int(walks))
    wrp = np.zeros(n + 1, np.int64)
    wcol = np.zeros(cap, np.int32)
    wcnt = np.zeros(cap, np.int32)
    st = _load().tsgo_random_walk_counts(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)), _ptr(Xd), d,
                                         int(walks), int(length), seed & (2 ** 64 - 1), _ptr(wrp), _ptr(wcol),
                                         _ptr(wcnt))
    _check(st, "random_walk_counts")
    m = int(wrp[n])
    return wrp, wcol[:m].copy(), wcnt[:m].copy()


def random_walk_P(n, row_ptr, col, X, walks, length, seed=0):
    """Joint P (Eq. 3) from the random-walk conditionals (Eq. 6) on the
    graph's neighbour structure; returns (rp, col, P) on the symmetrised
    structure of the walk pairs."""
    rp, cl = structure(n, row_ptr, col)
    wrp, wcol, wcnt = random_walk_counts(n, rp, cl, X, walks, length, seed)
    srp, scol = structure(n, wrp, wcol)
    pcond = np.zeros(max(1, scol.size))
    _check(_load().tsgo_random_walk_pcond(n, _ptr(wrp), _ptr(wcol if wcol.size else np.zeros(1, np.int32)),
                                          _ptr(wcnt if wcnt.size else np.zeros(1, np.int32)), int(walks), _ptr(srp),
                                          _ptr(scol if scol.size else np.zeros(1, np.int32)), _ptr(pcond)),
           "random_walk_pcond")
    P, _ = joint_P(n, srp, scol, pcond[: scol.size])
    return srp, scol, P


def repulsion_all(Y, threads=None, i0=0, i1=None):
    """Rows [i0, i1) (default all) of repulsion_rows, split over threads
    (ctypes drops the GIL).

    The split only partitions rows; each row is still the plain loop.
    Returns (F_rep, zrow) for those rows.
    """
    Yd = _c(Y, np.float64)
    n = Yd.shape[0]
    i1 = n if i1 is None else i1
    threads = threads or os.cpu_count() or 1
    bounds = np.linspace(i0, i1, 4 * threads + 1).astype(int)
    F = np.zeros((i1 - i0, 2))
    zr = np.zeros(i1 - i0)

    def work(k):
        a, b = int(bounds[k]), int(bounds[k + 1])
        if b > a:
            F[a - i0:b - i0], zr[a - i0:b - i0] = repulsion_rows(Yd, a, b)

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(work, range(len(bounds) - 1)))
    return F, zr


def attraction_rows(n, rp, col, P, Y, rows):
    rp, col, P, Yd = _c(rp, np.int64), _c(col, np.int32), _c(P, np.float64), _c(Y, np.float64)
    rows = _c(rows, np.int32)
    F = np.zeros((max(1, rows.size), 2))
    _check(_load().tsgo_attraction_rows(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)),
                                        _ptr(P if P.size else np.zeros(1)), _ptr(Yd), _ptr(rows), rows.size,
                                        _ptr(F)), "attraction_rows")
    return F[: rows.size]


def auto_learning_rate(n: int, early_exag: float) -> float:
    """eta = max(n / early_exag / 4, 50) (the published t-SNE rule; the paper gives none)."""
    return max(n / early_exag / 4.0, 50.0)


def optimize(n, rp, col, P, Y, n_iter, *, upd=None, gains=None, t0=0, early_exag=12.0, ee_iters=250,
             momentum0=0.5, momentum1=0.8, learning_rate=None, min_gain=0.01):
    """Runs n_iter iterations of the gradient-descent schedule; returns (Y, upd, gains)."""
    rp, col, P = _c(rp, np.int64), _c(col, np.int32), _c(P, np.float64)
    Yd = np.array(Y, dtype=np.float64, order="C", copy=True)
    u = np.zeros((n, 2)) if upd is None else np.array(upd, dtype=np.float64, order="C", copy=True)
    g = np.ones((n, 2)) if gains is None else np.array(gains, dtype=np.float64, order="C", copy=True)
    eta = auto_learning_rate(n, early_exag) if (learning_rate is None or learning_rate <= 0) else learning_rate
    st = _load().tsgo_optimize(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)),
                               _ptr(P if P.size else np.zeros(1)), _ptr(Yd), _ptr(u), _ptr(g), int(t0), int(n_iter),
                               float(early_exag), int(ee_iters), float(momentum0), float(momentum1), float(eta),
                               float(min_gain))
    _check(st, "optimize")
    return Yd, u, g


def default_l0(num_edges: int) -> int:
    """l0 = sqrt(|E|) (Sec. 2.3); distances are integers, so floor(sqrt(|E|))."""
    import math

    return int(math.isqrt(int(num_edges)))


def shortest_path_embedding(n, rp, col, targets, l0):
    """ShortestPath embedding (Eq. 8) on a symmetric CSR: n x d FP64."""
    rp, col = _c(rp, np.int64), _c(col, np.int32)
    tg = _c(targets, np.int32)
    X = np.zeros((n, tg.size))
    _check(_load().tsgo_shortest_path(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)), _ptr(tg),
                                      tg.size, int(l0), _ptr(X)), "shortest_path")
    return X


def bfs_knn(n, rp, col, k):
    """BFS k-nearest lists (Eq. 7) on a sorted structure: (out n x k, cnt n)."""
    rp, col = _c(rp, np.int64), _c(col, np.int32)
    out = np.full((n, k), -1, np.int32)
    cnt = np.zeros(n, np.int32)
    _check(_load().tsgo_bfs_knn(n, _ptr(rp), _ptr(col if col.size else np.zeros(1, np.int32)), int(k), _ptr(out),
                                _ptr(cnt)), "bfs_knn")
    return out, cnt


def knn_structure(n, row_ptr, col, k):
    """Neighbour structure with k_nn = k: BFS lists of the graph's structure,
    symmetrised by union (Eq. 7 read with k nodes per list)."""
    srp, scol = structure(n, row_ptr, col)
    out, cnt = bfs_knn(n, srp, scol, k)
    rows = np.repeat(np.arange(n), cnt)
    lists = np.concatenate([out[i, :cnt[i]] for i in range(n)]) if n else np.zeros(0, np.int32)
    krp = np.zeros(n + 1, np.int64)
    krp[1:] = np.cumsum(cnt)
    return structure(n, krp, lists.astype(np.int32))

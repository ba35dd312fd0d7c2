"""Seeded synthetic inputs for the t-SGNE layout loop.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It holds no arithmetic of the layout method itself: it only draws
graphs (stochastic block models), high-dimensional embeddings and initial
layouts from a counter-based generator, so that both sides of every parity
check receive bit-identical inputs on any machine and any numpy version.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in counter mode: the i-th draw of a
stream is ``mix(key + (i + 1) * GAMMA)`` with the published finaliser ``mix``.
Normals come from the Box-Muller transform.

Workload recipes (the paper's LFR / network-repository graphs are not
available, so these stand in for them):

* ``sbm_equal``: n nodes in equal blocks, every pair an independent Bernoulli
  draw with p_in inside a block and p_out across blocks.
* ``sbm_zipf``: block sizes proportional to r^-s (r = 1..B), a fixed number of
  distinct intra-block edges per block proportional to its size, then a
  fraction of edges rewired to a uniform endpoint (noise).
* ``block_embedding``: x_i = c_{b(i)} + eps_i with c_b ~ N(0, sc^2 I),
  eps_i ~ N(0, I).
* ``y_init``: Y0 ~ N(0, sigma^2 I) in 2-D, sigma = 1e-4.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64",
    "uniform",
    "normal",
    "Graph",
    "csr_from_edges",
    "sbm_equal",
    "sbm_zipf",
    "block_embedding",
    "y_init",
    "spread_layout",
    "random_graph",
    "workload",
    "poisson_arrivals",
    "log_uniform_ints",
    "sbm_mixed_batch",
    "rmat",
    "induced_bfs_ball",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

# stream identifiers: one per purpose so that draws never overlap
S_EDGE, S_REWIRE_PICK, S_REWIRE_DST, S_CENTRE, S_NOISE, S_YINIT, S_MISC = range(1, 8)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    """Per-(seed, stream) key: the mix of a combination of both."""
    k = (int(seed) * 0x632BE59BD9B4E019 + int(stream) * 0x8CB92BA72F3D8DD7 + 0x1234567) & _MASK64
    return _mix(np.array([k], dtype=np.uint64))[0]


def splitmix64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of stream ``stream`` as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(_key(seed, stream) + i * _GAMMA)


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    u = splitmix64(seed, stream, start, count) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller; draw k uses uniforms 2k and 2k+1."""
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * (start // 2), 2 * m + 2)
    u1 = 1.0 - u[0::2][: m + 1]  # (0, 1]
    u2 = u[1::2][: m + 1]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * (m + 1))
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    off = start - 2 * (start // 2)
    return z[off : off + count]


class Graph:
    """Undirected graph as CSR with both directions stored.

    row_ptr int64[n+1], col int32[m]; ``labels`` int32[n] are the planted
    blocks (or -1 when the generator plants none).
    """

    def __init__(self, n: int, row_ptr: np.ndarray, col: np.ndarray, labels: np.ndarray | None = None):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.labels = (
            np.ascontiguousarray(labels, dtype=np.int32) if labels is not None else np.full(n, -1, np.int32)
        )

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def __repr__(self) -> str:
        return f"Graph(n={self.n}, m={self.m})"


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """CSR holding each listed pair in both directions, rows sorted by column."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    # one int64 key per directed pair (row major), sorted: rows in order,
    # columns ascending within a row
    key = np.concatenate([u * n + v, v * n + u])
    key.sort()
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(key // n, minlength=n))
    return row_ptr, (key % n).astype(np.int32)


def _equal_blocks(n: int, blocks: int) -> np.ndarray:
    sizes = np.full(blocks, n // blocks, dtype=np.int64)
    sizes[: n % blocks] += 1
    return sizes


def _labels_from_sizes(sizes: np.ndarray) -> np.ndarray:
    return np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)


def sbm_equal(n: int, blocks: int, p_in: float, p_out: float, seed: int = 0) -> Graph:
    """Stochastic block model with equal blocks; each pair i<j drawn once."""
    sizes = _equal_blocks(n, blocks)
    labels = _labels_from_sizes(sizes)
    iu, ju = np.triu_indices(n, k=1)
    p = np.where(labels[iu] == labels[ju], p_in, p_out)
    keep = uniform(seed, S_EDGE, 0, iu.size) < p
    rp, col = csr_from_edges(n, iu[keep], ju[keep])
    return Graph(n, rp, col, labels)


def zipf_sizes(n: int, blocks: int, s: float) -> np.ndarray:
    """Block sizes proportional to r^-s, largest-remainder rounded to sum n."""
    w = np.arange(1, blocks + 1, dtype=np.float64) ** (-s)
    raw = n * w / w.sum()
    sizes = np.floor(raw).astype(np.int64)
    rem = n - int(sizes.sum())
    order = np.argsort(-(raw - sizes), kind="stable")
    sizes[order[:rem]] += 1
    return sizes


def _distinct_pairs(seed: int, stream: int, lo: int, size: int, count: int, counter0: int) -> tuple[np.ndarray, int]:
    """``count`` distinct unordered pairs inside [lo, lo+size), as keys u*2^32+v (u<v)."""
    have = np.empty(0, dtype=np.int64)
    ctr = counter0
    while have.size < count:
        need = count - have.size
        draw = int(need * 1.2) + 16
        r = splitmix64(seed, stream, ctr, 2 * draw)
        ctr += 2 * draw
        a = (r[0::2] % np.uint64(size)).astype(np.int64) + lo
        b = (r[1::2] % np.uint64(size)).astype(np.int64) + lo
        ok = a != b
        a, b = a[ok], b[ok]
        keys = np.minimum(a, b) * (1 << 32) + np.maximum(a, b)
        # first occurrence order keeps the result independent of set internals
        allk = np.concatenate([have, keys])
        _, first = np.unique(allk, return_index=True)
        first.sort()
        allk = allk[first]
        have = allk[:count]
    return have, ctr


def sbm_zipf(
    n: int,
    blocks: int,
    edges: int,
    zipf_s: float = 1.2,
    rewire: float = 0.10,
    seed: int = 0,
) -> Graph:
    """Zipf-sized stochastic block model with a fraction of edges rewired."""
    sizes = zipf_sizes(n, blocks, zipf_s)
    labels = _labels_from_sizes(sizes)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    keys = []
    ctr = 0
    for b in range(blocks):
        nb = int(sizes[b])
        want = int(round(edges * nb / n))
        want = min(want, nb * (nb - 1) // 2)
        if want <= 0:
            continue
        k, ctr = _distinct_pairs(seed, S_EDGE, int(starts[b]), nb, want, ctr)
        keys.append(k)
    keys = np.concatenate(keys)
    ne = keys.size
    n_rw = int(round(rewire * ne))
    if n_rw > 0:
        pick = np.argsort(splitmix64(seed, S_REWIRE_PICK, 0, ne), kind="stable")[:n_rw]
        pick.sort()
        keep_mask = np.ones(ne, dtype=bool)
        keep_mask[pick] = False
        kept = keys[keep_mask]
        src = keys[pick] >> 32  # first endpoint stays
        pending = np.arange(n_rw)
        new_keys = np.full(n_rw, -1, dtype=np.int64)
        taken = np.sort(kept)
        ctr = 0
        while pending.size:
            r = splitmix64(seed, S_REWIRE_DST, ctr, pending.size)
            ctr += pending.size
            dst = (r % np.uint64(n)).astype(np.int64)
            s = src[pending]
            cand = np.minimum(s, dst) * (1 << 32) + np.maximum(s, dst)
            ok = dst != s
            pos = np.searchsorted(taken, cand)
            pos = np.minimum(pos, taken.size - 1)
            ok &= taken[pos] != cand
            # among proposals of this round keep the first of equal keys
            idx = np.nonzero(ok)[0]
            _, first = np.unique(cand[idx], return_index=True)
            acc = np.zeros(pending.size, dtype=bool)
            acc[idx[first]] = True
            new_keys[pending[acc]] = cand[acc]
            taken = np.sort(np.concatenate([taken, cand[acc]]))
            pending = pending[~acc]
        keys = np.concatenate([kept, new_keys])
    u = keys >> 32
    v = keys & ((1 << 32) - 1)
    rp, col = csr_from_edges(n, u, v)
    return Graph(n, rp, col, labels)


def block_embedding(labels: np.ndarray, d: int, centre_std: float = 2.0, seed: int = 0) -> np.ndarray:
    """x_i = c_{b(i)} + eps_i, c_b ~ N(0, centre_std^2 I), eps ~ N(0, I); float32 n x d."""
    labels = np.asarray(labels)
    nb = int(labels.max()) + 1 if labels.size else 0
    centres = centre_std * normal(seed, S_CENTRE, 0, nb * d).reshape(nb, d)
    n = labels.size
    x = normal(seed, S_NOISE, 0, n * d).reshape(n, d)
    x += centres[labels]
    return x.astype(np.float32)


def y_init(n: int, sigma: float = 1e-4, seed: int = 0) -> np.ndarray:
    """Initial layout Y0 ~ N(0, sigma^2 I), float32 n x 2."""
    return (sigma * normal(seed, S_YINIT, 0, 2 * n)).astype(np.float32).reshape(n, 2)


def spread_layout(labels: np.ndarray, scale: float = 20.0, jitter: float = 1.0, seed: int = 0) -> np.ndarray:
    """A clustered 2-D layout of the size t-SNE reaches after convergence.

    Block centres ~ N(0, scale^2 I), points = centre + N(0, jitter^2 I).
    Used as a fixed Y for gradient parity away from the tiny initial scale.
    """
    labels = np.asarray(labels)
    nb = int(labels.max()) + 1 if labels.size else 1
    c = scale * normal(seed, S_MISC, 0, 2 * nb).reshape(nb, 2)
    y = c[np.maximum(labels, 0)] + jitter * normal(seed, S_MISC, 2 * nb + 2, 2 * labels.size).reshape(-1, 2)
    return y.astype(np.float32)


def random_graph(n: int, mean_deg: float, seed: int = 0) -> Graph:
    """Erdos-Renyi-like graph with ~n*mean_deg/2 distinct edges (small tests)."""
    want = int(round(n * mean_deg / 2))
    want = min(want, n * (n - 1) // 2)
    if want == 0 or n < 2:
        return Graph(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
    k, _ = _distinct_pairs(seed, S_EDGE, 0, n, want, 0)
    rp, col = csr_from_edges(n, k >> 32, k & ((1 << 32) - 1))
    return Graph(n, rp, col)


def workload(name: str, seed: int = 0):
    """The named synthetic workloads: returns (graph, X).

    ``sbm2k``: 2,000 nodes, 10 equal blocks, p_in 0.05, p_out 0.0005, 128-d X.
    ``zipf300k``: 300,000 nodes, 50 Zipf(1.2) blocks, 1,000,000 edges before
    rewiring, 10 % rewired, 128-d X.
    ``zipf100k``: the same recipe at 100,000 nodes and 333,333 edges (a
    smaller case of the same kernels, for profiling).
    ``zipf3m``: the same recipe at the scale of the paper's largest LFR graph
    (3,000,000 nodes, 4,937,941 edges: mean degree 3.3), 200 blocks, 64-d X.
    ``zipf4m``: the same recipe at the size of the paper's largest real graph
    (3,997,962 nodes, 34,681,189 edges: mean degree 17.3), 500 blocks, 32-d X.
    """
    if name == "sbm2k":
        g = sbm_equal(2000, 10, 0.05, 0.0005, seed=seed)
        return g, block_embedding(g.labels, 128, seed=seed)
    if name == "zipf300k":
        g = sbm_zipf(300_000, 50, 1_000_000, 1.2, 0.10, seed=seed)
        return g, block_embedding(g.labels, 128, seed=seed)
    if name == "zipf100k":
        g = sbm_zipf(100_000, 50, 333_333, 1.2, 0.10, seed=seed)
        return g, block_embedding(g.labels, 128, seed=seed)
    if name == "zipf3m":
        g = sbm_zipf(3_000_000, 200, 4_937_941, 1.2, 0.10, seed=seed)
        return g, block_embedding(g.labels, 64, seed=seed)
    if name == "zipf4m":
        g = sbm_zipf(3_997_962, 500, 34_681_189, 1.2, 0.10, seed=seed)
        return g, block_embedding(g.labels, 32, seed=seed)
    raise KeyError(name)


S_ARRIVAL, S_SIZES = 97, 98


def poisson_arrivals(count: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps of mean 1/rate."""
    u = uniform(seed, S_ARRIVAL, 0, count)
    return np.cumsum(-np.log1p(-u) / rate)


def log_uniform_ints(count: int, lo: int, hi: int, seed: int = 0, stream: int = S_SIZES) -> np.ndarray:
    """Integers log-uniform in [lo, hi]."""
    u = uniform(seed, stream, 0, count)
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64).clip(lo, hi)


def sbm_mixed_batch(count: int, n_lo: int, n_hi: int, deg_lo: float, deg_hi: float, blocks_lo: int, blocks_hi: int,
                    d: int, seed: int = 0):
    """``count`` block-model graphs for batched runs: n log-uniform in
    [n_lo, n_hi], mean degree uniform in [deg_lo, deg_hi], blocks uniform in
    [blocks_lo, blocks_hi] (equal sizes), 10 % of edges rewired, d-dimensional
    block-centre embeddings.  Returns a list of (Graph, X)."""
    ns = log_uniform_ints(count, n_lo, n_hi, seed=seed)
    degs = deg_lo + (deg_hi - deg_lo) * uniform(seed, S_SIZES + 1, 0, count)
    nbs = blocks_lo + np.floor((blocks_hi - blocks_lo + 1) * uniform(seed, S_SIZES + 2, 0, count)).astype(int)
    out = []
    for k in range(count):
        n = int(ns[k])
        nb = int(min(nbs[k], max(1, n // 8)))
        edges = int(round(n * degs[k] / 2))
        g = sbm_zipf(n, nb, edges, zipf_s=0.0, rewire=0.10, seed=seed * 100003 + k)
        out.append((g, block_embedding(g.labels, d, seed=seed * 100003 + k)))
    return out


S_RMAT = 99


def rmat(scale: int, edges: int, a: float = 0.57, b: float = 0.19, c: float = 0.19, d_emb: int = 64,
         community_bits: int = 6, seed: int = 0, chunk: int = 1 << 22):
    """R-MAT graph (Chakrabarti, Zhan, Faloutsos 2004) with 2^scale nodes:
    each edge descends ``scale`` levels choosing quadrant (0,0), (0,1), (1,0),
    (1,1) with probabilities a, b, c, 1-a-b-c (one 32-bit uniform per level,
    two per SplitMix64 draw); draws continue until ``edges`` distinct
    undirected non-loop edges exist, keeping first occurrences in draw order.
    Communities are the top ``community_bits`` bits of the node id (the first
    levels of the recursion); X = community centre N(0, 4I) + N(0, I) in
    ``d_emb`` dimensions.  Returns (Graph, X)."""
    n = 1 << scale
    half = (scale + 1) // 2
    ta, tab, tabc = (np.uint64(int(x * 2 ** 32)) for x in (a, a + b, a + b + c))
    keys_all = []
    have = 0
    ctr = 0
    while True:
        m = chunk
        r = splitmix64(seed, S_RMAT, ctr, m * half).reshape(half, m)
        ctr += m * half
        src = np.zeros(m, dtype=np.int64)
        dst = np.zeros(m, dtype=np.int64)
        for lvl in range(scale):
            w = r[lvl // 2]
            u32 = (w >> np.uint64(32)) if (lvl & 1) == 0 else (w & np.uint64(0xFFFFFFFF))
            bit_s = u32 >= tab
            bit_d = ((u32 >= ta) & (u32 < tab)) | (u32 >= tabc)
            src = (src << 1) | bit_s
            dst = (dst << 1) | bit_d
        ok = src != dst
        keys_all.append(np.minimum(src[ok], dst[ok]) * n + np.maximum(src[ok], dst[ok]))
        have += int(ok.sum())
        if have < edges:
            continue
        allk = np.concatenate(keys_all)
        _, first = np.unique(allk, return_index=True)
        if first.size >= edges:
            first.sort()
            keys = allk[first[:edges]]
            break
        keys_all = [allk]
    u_, v_ = keys // n, keys % n
    rp, col = csr_from_edges(n, u_, v_)
    labels = (np.arange(n) >> (scale - community_bits)).astype(np.int32)
    return Graph(n, rp, col, labels), block_embedding(labels, d_emb, seed=seed)


def induced_bfs_ball(g: Graph, size: int, start: int | None = None):
    """Nodes of a BFS ball (levels in order, neighbours in ascending id) from
    ``start`` (default: the highest-degree node), truncated at ``size``, and
    the induced subgraph on them (ids renumbered in that order).
    Returns (nodes int64[k], Graph)."""
    deg = np.diff(g.row_ptr)
    s = int(np.argmax(deg)) if start is None else int(start)
    seen = np.zeros(g.n, dtype=bool)
    seen[s] = True
    order = [s]
    head = 0
    while head < len(order) and len(order) < size:
        v = order[head]
        head += 1
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        for w in np.sort(nb):
            if not seen[w]:
                seen[w] = True
                order.append(int(w))
                if len(order) >= size:
                    break
    nodes = np.array(order, dtype=np.int64)
    remap = np.full(g.n, -1, dtype=np.int64)
    remap[nodes] = np.arange(nodes.size)
    rows = np.repeat(np.arange(g.n), deg)
    keep = (remap[rows] >= 0) & (remap[g.col] >= 0) & (rows < g.col)
    rp, col = csr_from_edges(nodes.size, remap[rows[keep]], remap[g.col[keep]])
    return nodes, Graph(nodes.size, rp, col, g.labels[nodes])

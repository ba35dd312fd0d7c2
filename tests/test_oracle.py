"""Pins for the FP64 oracle (CPU only).

Each test checks the oracle against something other than itself: brute force
on tiny inputs, closed forms, finite differences, library routines, or
invariants that the definitions of the paper fix (Li, Xiao, Zhou, arXiv
2310.11186, Sec. 2.1-2.2, Eqs. 2-5 and 7).  The cases are chosen so that a
dropped term, a wrong sign, a wrong index or a transposed operand in the
oracle fails at least one of them.
"""

import math

import numpy as np
import pytest

import oracle
import tsgne_synth as synth


def _rand_csr(n, m, seed, loops=True, dups=True):
    """An arbitrary (asymmetric, unsorted, duplicated, looped) CSR."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    dst = rng.integers(0, n, m)
    if not loops:
        ok = src != dst
        src, dst = src[ok], dst[ok]
    if dups and src.size:
        src = np.concatenate([src, src[: m // 4]])
        dst = np.concatenate([dst, dst[: m // 4]])
    perm = rng.permutation(src.size)
    src, dst = src[perm], dst[perm]
    order = np.argsort(src, kind="stable")  # rows grouped, columns unsorted
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    return rp, dst.astype(np.int32)


def _dense_P(n, rp, col, P):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, col[rp[i]:rp[i + 1]]] = P[rp[i]:rp[i + 1]]
    return D


# ----------------------------------------------------------------- structure


@pytest.mark.parametrize("n,m,seed", [(1, 0, 0), (2, 1, 1), (7, 20, 2), (40, 150, 3), (100, 50, 4)])
def test_structure_is_set_union(n, m, seed):
    """Eq. 7 with graph-edge neighbours: N(i) = {j != i : (i,j) or (j,i) in G}."""
    rp, col = _rand_csr(n, m, seed)
    orp, ocol = oracle.structure(n, rp, col)
    want = [set() for _ in range(n)]
    for i in range(n):
        for j in col[rp[i]:rp[i + 1]]:
            if j != i:
                want[i].add(int(j))
                want[j].add(i)
    for i in range(n):
        got = ocol[orp[i]:orp[i + 1]].tolist()
        assert got == sorted(want[i])
    assert orp[0] == 0 and orp[-1] == ocol.size


def test_structure_rejects_bad_csr():
    good_rp = np.array([0, 1, 2], np.int64)
    assert oracle.check_csr(2, good_rp, np.array([1, 0], np.int32)) == 0
    assert oracle.check_csr(2, np.array([1, 1, 2], np.int64), np.array([1, 0], np.int32)) == -2
    assert oracle.check_csr(2, np.array([0, 2, 1], np.int64), np.array([1, 0], np.int32)) == -2
    assert oracle.check_csr(2, good_rp, np.array([1, 2], np.int32)) == -2
    assert oracle.check_csr(2, good_rp, np.array([-1, 0], np.int32)) == -2
    with pytest.raises(oracle.OracleError):
        oracle.structure(2, good_rp, np.array([1, 5], np.int32))


def test_transpose_slots():
    rp, col = _rand_csr(30, 90, 7)
    srp, scol = oracle.structure(30, rp, col)
    t = oracle.transpose_slots(30, srp, scol)
    rows = np.repeat(np.arange(30), np.diff(srp))
    # entry t[e] sits in row col[e] and points back at row(e)
    assert np.array_equal(scol[t], rows)
    assert np.array_equal(rows[t], scol)
    assert np.array_equal(t[t], np.arange(scol.size))


# ------------------------------------------------------ conditional affinity


def _graph_and_X(n=60, deg=12.0, d=16, seed=5):
    g = synth.random_graph(n, deg, seed=seed)
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, d)).astype(np.float32)
    return g, X


@pytest.mark.parametrize("perp", [2.0, 3.0, 5.0, 8.5])
def test_bisection_reaches_target_entropy(perp):
    """Sec. 2.1: Perp(P_i) = 2^{H(P_i)} equals the user value, H in bits."""
    g, X = _graph_and_X()
    rp, col = oracle.structure(g.n, g.row_ptr, g.col)
    pc, beta, iters = oracle.cond_affinity(g.n, rp, col, X, perp)
    checked = 0
    for i in range(g.n):
        p = pc[rp[i]:rp[i + 1]]
        k = p.size
        if k == 0:
            continue
        assert abs(p.sum() - 1.0) < 1e-12
        if k <= perp:
            assert np.all(p == 1.0 / k)  # saturated rows are uniform
            continue
        H_bits = -(p * np.log2(p)).sum()
        assert abs(2.0 ** H_bits - perp) / perp < 2e-5
        checked += 1
    assert checked > 10


def test_affinity_is_gaussian_in_squared_distance():
    """Eq. 2: ln p_{j|i} - ln p_{k|i} = -beta_i (|x_i-x_j|^2 - |x_i-x_k|^2)."""
    g, X = _graph_and_X(d=7)
    rp, col = oracle.structure(g.n, g.row_ptr, g.col)
    pc, beta, _ = oracle.cond_affinity(g.n, rp, col, X, 3.0)
    X64 = X.astype(np.float64)
    for i in range(g.n):
        nb = col[rp[i]:rp[i + 1]]
        if nb.size <= 3:
            continue
        d2 = ((X64[nb] - X64[i]) ** 2).sum(axis=1)
        lp = np.log(pc[rp[i]:rp[i + 1]])
        np.testing.assert_allclose(lp - lp[0], -beta[i] * (d2 - d2[0]), rtol=1e-9, atol=1e-9)


def test_bisection_two_level_row_against_brentq():
    """Row with k1 neighbours at distance a and k2 at distance b: beta solves
    H(beta) = ln perp, cross-checked with scipy's brentq on the closed form."""
    brentq = pytest.importorskip("scipy.optimize").brentq
    k1, k2, perp = 3, 9, 6.0
    n = 1 + k1 + k2
    # star graph around node 0; node positions on a line so distances are exact
    X = np.zeros((n, 1))
    X[1:1 + k1, 0] = 1.0   # distance^2 = 1
    X[1 + k1:, 0] = 2.0    # distance^2 = 4
    rp, col = synth.csr_from_edges(n, np.zeros(k1 + k2, np.int64), np.arange(1, n))
    pc, beta, _ = oracle.cond_affinity(n, rp, col, X, perp, tol=1e-12, max_iter=200)

    def H(bt):  # two-level row entropy in nats, shift by the smaller distance
        e = math.exp(-bt * 3.0)
        S = k1 + k2 * e
        return math.log(S) + bt * (k2 * 3.0 * e) / S

    root = brentq(lambda bt: H(bt) - math.log(perp), 1e-9, 50.0, xtol=1e-14)
    assert abs(beta[0] - root) < 1e-8
    p_near = 1.0 / (k1 + k2 * math.exp(-root * 3.0))
    np.testing.assert_allclose(pc[rp[0]:rp[0] + k1], p_near, rtol=1e-9)


# --------------------------------------------------------------- joint P


def test_joint_P_symmetric_normalised():
    """Eq. 3: p_ij = p_ji, sum P = 1, p > 0 exactly on the structure."""
    g, X = _graph_and_X(n=80)
    rp, col, P = oracle.build_P(g.n, g.row_ptr, g.col, X, 3.0)
    t = oracle.transpose_slots(g.n, rp, col)
    assert np.all(P > 0)
    assert np.array_equal(P, P[t])
    assert abs(P.sum() - 1.0) < 1e-12


def test_joint_P_uniform_rows_closed_form():
    """All rows saturated: p_ij = (1/deg_i + 1/deg_j) / T, T = 2 * #non-isolated."""
    g = synth.sbm_equal(120, 4, 0.12, 0.01, seed=3)
    X = synth.block_embedding(g.labels, 8, seed=3)
    rp, col, P = oracle.build_P(g.n, g.row_ptr, g.col, X, 1000.0)
    deg = np.diff(rp)
    T = 2.0 * np.count_nonzero(deg)
    rows = np.repeat(np.arange(g.n), deg)
    np.testing.assert_allclose(P, (1.0 / deg[rows] + 1.0 / deg[col]) / T, rtol=1e-13)


def test_joint_P_isolated_nodes_keep_sum_one():
    rp = np.array([0, 1, 2, 2, 2], np.int64)  # 0-1 edge, nodes 2, 3 isolated
    col = np.array([1, 0], np.int32)
    X = np.arange(8, dtype=np.float32).reshape(4, 2)
    srp, scol, P = oracle.build_P(4, rp, col, X, 30.0)
    assert np.allclose(P, [0.5, 0.5])


# ------------------------------------------------------------- Z, KL, grad


def test_Z_two_points_and_dense():
    """Eq. 4 denominator over ordered pairs."""
    Y = np.array([[0.0, 0.0], [3.0, 4.0]])
    assert oracle.Z(Y) == pytest.approx(2.0 / 26.0, rel=1e-15)
    rng = np.random.default_rng(0)
    Y = rng.normal(scale=3.0, size=(50, 2))
    D2 = ((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    W = 1.0 / (1.0 + D2)
    np.fill_diagonal(W, 0.0)
    assert oracle.Z(Y) == pytest.approx(W.sum(), rel=1e-13)


def test_kl_two_nodes_is_zero():
    """2-node graph: p = q = 1/2 per ordered pair for any Y, KL = 0, g = 0."""
    rp, col = np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32)
    P = np.array([0.5, 0.5])
    for Y in ([[0.0, 0.0], [1.0, 2.0]], [[5.0, -3.0], [5.0, -3.0]]):
        v, _ = oracle.kl(2, rp, col, P, np.array(Y))
        assert abs(v) < 1e-15
        G, _ = oracle.gradient(2, rp, col, P, np.array(Y))
        assert np.abs(G).max() < 1e-15


def _path3(a):
    rp, col = synth.csr_from_edges(3, np.array([0, 1]), np.array([1, 2]))
    Y = np.array([[-a, 0.0], [0.0, 0.0], [a, 0.0]])
    return rp, col, Y


@pytest.mark.parametrize("a", [0.0, 0.3, 1.0, 2.5])
def test_kl_path3_closed_form(a):
    """Path 0-1-2, uniform rows: P has four entries 1/4 and
    KL(a) = ln(1 + (1+a^2) / (2 (1+4a^2))) at Y = (-a,0), (0,0), (a,0)."""
    rp, col, Y = _path3(a)
    X = np.zeros((3, 1), np.float32)
    srp, scol, P = oracle.build_P(3, rp, col, X, 30.0)
    assert np.allclose(P, 0.25)
    v, _ = oracle.kl(3, srp, scol, P, Y)
    assert v == pytest.approx(math.log(1 + (1 + a * a) / (2 * (1 + 4 * a * a))), rel=1e-13, abs=1e-15)
    G, _ = oracle.gradient(3, srp, scol, P, Y)
    # middle node: zero by symmetry; end node: half the derivative of KL(a)
    dkl = (-3 * a / (1 + 4 * a * a) ** 2) / (1 + (1 + a * a) / (2 * (1 + 4 * a * a)))
    assert np.abs(G[1]).max() < 1e-15
    assert G[2, 0] == pytest.approx(0.5 * dkl, rel=1e-12, abs=1e-15)
    assert G[0, 0] == pytest.approx(-0.5 * dkl, rel=1e-12, abs=1e-15)
    assert abs(G[0, 1]) < 1e-15 and abs(G[2, 1]) < 1e-15


def _small_case(n=30, seed=11, perp=3.0, scale=2.0):
    g = synth.random_graph(n, 6.0, seed=seed)
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 5)).astype(np.float32)
    rp, col, P = oracle.build_P(n, g.row_ptr, g.col, X, perp)
    Y = rng.normal(scale=scale, size=(n, 2))
    return rp, col, P, Y


def test_kl_dense_brute_force_and_invariances():
    """Eq. 5 from the full dense P and Q; KL >= 0; invariant to rigid motions."""
    rp, col, P, Y = _small_case()
    n = Y.shape[0]
    Pd = _dense_P(n, rp, col, P)
    D2 = ((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    W = 1.0 / (1.0 + D2)
    np.fill_diagonal(W, 0.0)
    Q = W / W.sum()
    m = Pd > 0
    want = (Pd[m] * np.log(Pd[m] / Q[m])).sum()
    v, _ = oracle.kl(n, rp, col, P, Y)
    assert v == pytest.approx(want, rel=1e-12)
    assert v > 0
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    v2, _ = oracle.kl(n, rp, col, P, Y @ R.T + np.array([3.0, -1.5]))
    assert v2 == pytest.approx(v, rel=1e-12)


@pytest.mark.parametrize("alpha", [1.0, 4.0, 12.0])
def test_gradient_matches_finite_differences(alpha):
    """g = d f / dY with f(Y) = -alpha sum_e p_e ln w_e + ln Z, which is KL(P||Q)
    up to a constant when alpha = 1 (Eq. 5); central differences in numpy."""
    rp, col, P, Y = _small_case()
    n = Y.shape[0]
    rows = np.repeat(np.arange(n), np.diff(rp))

    def f(Yv):
        D2 = ((Yv[:, None, :] - Yv[None, :, :]) ** 2).sum(-1)
        W = 1.0 / (1.0 + D2)
        np.fill_diagonal(W, 0.0)
        return -alpha * (P * np.log(W[rows, col])).sum() + math.log(W.sum())

    G, _ = oracle.gradient(n, rp, col, P, Y, alpha)
    FD = np.zeros_like(Y)
    for i in range(n):
        for c in range(2):
            h = 1e-6 * max(1.0, abs(Y[i, c]))
            Yp, Ym = Y.copy(), Y.copy()
            Yp[i, c] += h
            Ym[i, c] -= h
            FD[i, c] = (f(Yp) - f(Ym)) / (2 * h)
    assert np.linalg.norm(G - FD) / np.linalg.norm(FD) < 1e-6
    if alpha == 1.0:
        # the same derivative taken of the oracle's own KL
        i, c = 3, 1
        h = 1e-6
        Yp, Ym = Y.copy(), Y.copy()
        Yp[i, c] += h
        Ym[i, c] -= h
        d = (oracle.kl(n, rp, col, P, Yp)[0] - oracle.kl(n, rp, col, P, Ym)[0]) / (2 * h)
        assert G[i, c] == pytest.approx(d, rel=1e-6)


def test_gradient_sums_to_zero():
    """Pairwise antisymmetric forces: sum_i g_i = 0."""
    rp, col, P, Y = _small_case(n=50, seed=2)
    G, _ = oracle.gradient(50, rp, col, P, Y, 12.0)
    assert np.abs(G.sum(0)).max() < 1e-12 * np.abs(G).sum()


def test_row_splits_agree_with_gradient():
    """repulsion_rows / attraction_rows recombine into the gradient and Z."""
    rp, col, P, Y = _small_case(n=40, seed=9)
    n = 40
    G1, Z = oracle.gradient(n, rp, col, P, Y, 1.0)
    Fr, zr = oracle.repulsion_all(Y, threads=3)
    assert zr.sum() == pytest.approx(Z, rel=1e-14)
    Fa = oracle.attraction_rows(n, rp, col, P, Y, np.arange(n))
    np.testing.assert_allclose(4.0 * (Fa - Fr / Z), G1, rtol=1e-12, atol=1e-15)
    G5, _ = oracle.gradient(n, rp, col, P, Y, 5.0)
    np.testing.assert_allclose(G5 - G1, 16.0 * Fa, rtol=1e-10, atol=1e-14)


# --------------------------------------------------------------- optimiser


def test_optimizer_two_nodes_does_not_move():
    rp, col = np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32)
    Y0 = np.array([[0.1, -0.2], [0.3, 0.4]])
    # alpha = 1: p = q, the gradient vanishes up to rounding, nothing moves
    Y, u, g = oracle.optimize(2, rp, col, np.array([0.5, 0.5]), Y0, 5, ee_iters=0)
    np.testing.assert_allclose(Y, Y0, rtol=0, atol=1e-12)
    # alpha = 12: attraction dominates, the two points approach each other
    Y, u, g = oracle.optimize(2, rp, col, np.array([0.5, 0.5]), Y0, 1, learning_rate=1e-3)
    assert np.linalg.norm(Y[0] - Y[1]) < np.linalg.norm(Y0[0] - Y0[1])


def test_optimizer_hand_trace_path3():
    """Three iterations on the symmetric 3-node path, traced by hand with the
    closed-form gradient (alpha = 1 throughout, momentum 0.5, eta = 10):
        gains start at 1 and updates at 0; g*upd < 0 -> gain + 0.2 else
        gain * 0.8; upd = mu*upd - eta*gain*g; y += upd."""
    def g_end(a):  # d KL / d y_2x at half-width a (closed form above)
        return 0.5 * (-3 * a / (1 + 4 * a * a) ** 2) / (1 + (1 + a * a) / (2 * (1 + 4 * a * a)))

    eta, mu = 10.0, 0.5
    a0 = 0.05
    # t = 0: upd = 0 -> product 0 -> gain 0.8
    g0 = g_end(a0); gain1 = 0.8; u1 = -eta * gain1 * g0; a1 = a0 + u1
    # t = 1: g1 has the sign of g0 while u1 has the opposite one -> gain 1.0
    g1 = g_end(a1); assert g1 * u1 < 0; gain2 = gain1 + 0.2
    u2 = mu * u1 - eta * gain2 * g1; a2 = a1 + u2
    # t = 2
    g2 = g_end(a2); gain3 = gain2 + 0.2 if g2 * u2 < 0 else gain2 * 0.8
    u3 = mu * u2 - eta * gain3 * g2; a3 = a2 + u3
    rp, col, Y0 = _path3(a0)
    P = np.full(4, 0.25)
    Y, u, gains = oracle.optimize(3, rp, col, P, Y0, 3, early_exag=1.0, ee_iters=0, momentum0=mu,
                                  momentum1=mu, learning_rate=eta)
    assert Y[2, 0] == pytest.approx(a3, rel=1e-12)
    assert Y[0, 0] == pytest.approx(-a3, rel=1e-12)
    assert np.abs(Y[1]).max() < 1e-15 and np.abs(Y[:, 1]).max() < 1e-15
    assert gains[2, 0] == pytest.approx(gain3, rel=1e-14)
    assert gains[2, 1] == pytest.approx(0.8 ** 3, rel=1e-14)  # y-gradient stays 0
    assert u[2, 0] == pytest.approx(u3, rel=1e-12)


def test_optimizer_schedule_switches_at_ee_iters():
    """Splitting a run at any point gives the same trajectory (state = Y, upd,
    gains, t); the exaggeration phase differs from the plain phase."""
    rp, col, P, Y = _small_case(n=25, seed=4, scale=1e-2)
    full = oracle.optimize(25, rp, col, P, Y, 12, ee_iters=5, learning_rate=50.0)
    a = oracle.optimize(25, rp, col, P, Y, 7, ee_iters=5, learning_rate=50.0)
    b = oracle.optimize(25, rp, col, P, a[0], 5, upd=a[1], gains=a[2], t0=7, ee_iters=5, learning_rate=50.0)
    for x, y in zip(full, b):
        assert np.array_equal(x, y)
    no_ee = oracle.optimize(25, rp, col, P, Y, 12, ee_iters=0, learning_rate=50.0)
    assert not np.allclose(no_ee[0], full[0])


def test_auto_learning_rate():
    assert oracle.auto_learning_rate(2000, 12.0) == 50.0
    assert oracle.auto_learning_rate(300000, 12.0) == 6250.0


# -------------------------------------------------------- ShortestPath (Eq. 8)


def test_shortest_path_on_a_path_graph():
    """Path 0-1-...-9: the distance to target t is |i - t|, capped at l0 + 1."""
    n = 10
    rp, col = synth.csr_from_edges(n, np.arange(n - 1), np.arange(1, n))
    X = oracle.shortest_path_embedding(n, rp, col, [0, 4, 9], l0=5)
    i = np.arange(n)[:, None]
    want = np.abs(i - np.array([0, 4, 9])[None, :]).astype(float)
    want[want > 5] = 6
    assert np.array_equal(X, want)


def test_shortest_path_against_scipy_and_unreachable():
    sp = pytest.importorskip("scipy.sparse.csgraph")
    sps = pytest.importorskip("scipy.sparse")
    g = synth.random_graph(300, 2.5, seed=4)  # sparse: several components
    A = sps.csr_matrix((np.ones(g.col.size), g.col, g.row_ptr), shape=(g.n, g.n))
    targets = np.array([3, 50, 120, 299], np.int32)
    D = sp.shortest_path(A, unweighted=True, indices=targets).T
    l0 = oracle.default_l0(g.m // 2)
    want = np.where(np.isfinite(D) & (D <= l0), D, l0 + 1)
    X = oracle.shortest_path_embedding(g.n, g.row_ptr, g.col, targets, l0)
    assert np.array_equal(X, want)
    assert (X == l0 + 1).any()  # some nodes are unreachable or farther than l0


# ----------------------------------------------------- BFS-k neighbours (Eq. 7)


def _py_bfs_lists(n, rp, col, k):
    """Independent brute force: deque BFS with sorted neighbour scans."""
    from collections import deque

    lists = []
    for s in range(n):
        seen = {s}
        q = deque([s])
        found = []
        while q and len(found) < k:
            v = q.popleft()
            for w in sorted(col[rp[v]:rp[v + 1]].tolist()):
                if w not in seen:
                    seen.add(w)
                    q.append(w)
                    found.append(w)
                    if len(found) == k:
                        break
        lists.append(found)
    return lists


@pytest.mark.parametrize("n,deg,k", [(30, 3.0, 4), (80, 2.0, 10), (60, 8.0, 25)])
def test_bfs_knn_brute_force(n, deg, k):
    g = synth.random_graph(n, deg, seed=n + k)
    rp, col = oracle.structure(n, g.row_ptr, g.col)
    out, cnt = oracle.bfs_knn(n, rp, col, k)
    want = _py_bfs_lists(n, rp, col, k)
    for i in range(n):
        assert out[i, :cnt[i]].tolist() == want[i]


def test_bfs_knn_closed_forms():
    # path 0-1-...-9, k = 2: interior nodes get (i-1, i+1); ends get the next two
    n = 10
    rp, col = synth.csr_from_edges(n, np.arange(n - 1), np.arange(1, n))
    out, cnt = oracle.bfs_knn(n, rp, col, 2)
    assert out[0].tolist() == [1, 2] and out[9].tolist() == [8, 7] and out[4].tolist() == [3, 5]
    # star with centre 0 and 6 leaves, k = 3: centre -> 3 smallest leaves,
    # leaf -> centre then the 2 smallest other leaves
    rp, col = synth.csr_from_edges(7, np.zeros(6, np.int64), np.arange(1, 7))
    out, cnt = oracle.bfs_knn(7, rp, col, 3)
    assert out[0].tolist() == [1, 2, 3] and out[5].tolist() == [0, 1, 2]
    # a component smaller than k: the whole component
    rp, col = synth.csr_from_edges(5, np.array([0, 3]), np.array([1, 4]))
    out, cnt = oracle.bfs_knn(5, rp, col, 4)
    assert cnt.tolist() == [1, 1, 0, 1, 1]
    # symmetrised structure = union of the lists: 2 is in the lists of 0, 1, 3
    krp, kcol = oracle.knn_structure(10, *synth.csr_from_edges(10, np.arange(9), np.arange(1, 10)), 2)
    assert kcol[krp[0]:krp[1]].tolist() == [1, 2] and kcol[krp[2]:krp[3]].tolist() == [0, 1, 3]


# ------------------------------------------------ tree-code repulsion (extension)


def _exact_rep(Y):
    F, zr = oracle.repulsion_rows(Y, 0, Y.shape[0])
    return F, zr


@pytest.mark.parametrize("n", [1, 2, 31, 33, 1000])
def test_tree_theta0_equals_exact_sums(n):
    """theta = 0 accepts no node: every pair is summed exactly."""
    Y = np.random.default_rng(n).normal(size=(n, 2)).astype(np.float32)
    F, zr, Z = oracle.repulsion_tree(Y, 0.0)
    Fe, ze = _exact_rep(Y)
    # same terms in another order: FP64 rounding only
    assert np.abs(F - Fe).max() <= 1e-12 * max(np.abs(Fe).max(), 1e-300)
    assert np.allclose(zr, ze, rtol=1e-12)
    assert Z == pytest.approx(ze.sum(), rel=1e-12, abs=0.0)


def test_tree_far_cluster_is_one_monopole():
    """Two 32-point clusters 100 apart on the x axis: the root splits them
    (x's top cell bit differs), each is one group, and each sees the other
    as a single node of weight 32 at its centre of mass."""
    rng = np.random.default_rng(7)
    A = rng.uniform(-0.5, 0.5, size=(32, 2))
    B = rng.uniform(-0.5, 0.5, size=(32, 2)) + [100.0, 0.0]
    Y = np.concatenate([B, A]).astype(np.float32)  # input order does not matter
    Yd = Y.astype(np.float64)
    F, zr, Z = oracle.repulsion_tree(Y, 0.5)
    for own, other in ((slice(32, 64), slice(0, 32)), (slice(0, 32), slice(32, 64))):
        c = Yd[other].mean(0)
        for i in range(own.start, own.stop):
            d = Yd[own] - Yd[i]
            w = 1.0 / (1.0 + (d ** 2).sum(1))
            m = np.arange(own.start, own.stop) != i
            e = Yd[i] - Yd[own][m]
            f_in = ((w[m] ** 2)[:, None] * e).sum(0)
            wc = 1.0 / (1.0 + ((Yd[i] - c) ** 2).sum())
            f = f_in + 32 * wc ** 2 * (Yd[i] - c)
            z = w[m].sum() + 32 * wc
            assert np.allclose(F[i], f, rtol=1e-6, atol=1e-12), (i, F[i], f)
            assert zr[i] == pytest.approx(z, rel=1e-9)
    # and the monopole differs from the exact far-field sum (it is an approximation)
    Fe, _ = _exact_rep(Y)
    assert not np.allclose(F, Fe, rtol=1e-9, atol=0)


def test_tree_error_shrinks_with_theta():
    n = 5000
    lab = (np.arange(n) % 7).astype(np.int32)
    Y = synth.spread_layout(lab, scale=20.0, seed=1).astype(np.float32)
    Fe, ze = _exact_rep(Y)
    errs, zerr = [], []
    for th in (0.1, 0.25, 0.5, 1.0):
        F, _, Z = oracle.repulsion_tree(Y, th)
        errs.append(np.linalg.norm(F - Fe) / np.linalg.norm(Fe))
        zerr.append(abs(Z - ze.sum()) / ze.sum())
    assert all(a < b for a, b in zip(errs, errs[1:])), errs
    assert errs[0] < 5e-4 and errs[2] < 1e-2 and zerr[2] < 5e-3, (errs, zerr)


def test_tree_coincident_points():
    """200 points on one spot: their nodes have r = 0, so accepting them is
    exact; duplicates are split by position, not by coordinates."""
    rng = np.random.default_rng(3)
    Y = np.concatenate([np.full((200, 2), 1.0), rng.normal(scale=5.0, size=(300, 2))]).astype(np.float32)
    Fe, ze = _exact_rep(Y)
    for th in (0.0, 0.5):
        F, zr, Z = oracle.repulsion_tree(Y, th)
        assert np.all(np.isfinite(F))
        assert np.linalg.norm(F - Fe) / np.linalg.norm(Fe) < (1e-12 if th == 0 else 1e-2)
        assert abs(Z - ze.sum()) / ze.sum() < (1e-12 if th == 0 else 5e-3)


def test_tree_gradient_reduces_to_exact_at_theta0():
    g = synth.random_graph(300, 5.0, seed=2)
    X = synth.block_embedding((np.arange(300) % 4).astype(np.int32), 8, seed=2)
    rp, col, P = oracle.build_P(300, g.row_ptr, g.col, X, 5.0)
    Y = synth.spread_layout((np.arange(300) % 4).astype(np.int32), scale=10.0, seed=2).astype(np.float32)
    for alpha in (1.0, 12.0):
        Gt, Zt = oracle.gradient_tree(300, rp, col, P, Y, alpha, theta=0.0)
        Ge, Ze = oracle.gradient(300, rp, col, P, Y.astype(np.float64), alpha)
        assert np.abs(Gt - Ge).max() <= 1e-12 * np.abs(Ge).max()
        assert Zt == pytest.approx(Ze, rel=1e-12)
    # theta > 0 moves the repulsive part only: alpha-scaled attraction is shared
    G1, Z1 = oracle.gradient_tree(300, rp, col, P, Y, 1.0, theta=0.8)
    G2, Z2 = oracle.gradient_tree(300, rp, col, P, Y, 2.0, theta=0.8)
    Fa = oracle.attraction_rows(300, rp, col, P, Y.astype(np.float64), np.arange(300))
    assert Z1 == Z2 and np.allclose(G2 - G1, 4 * Fa, rtol=1e-10, atol=1e-15)


def test_tree_outliers_keep_resolution():
    """A few points 400x farther out than the bulk stretch the bounding
    square; 32-bit cells per axis still separate the bulk, so the error at
    theta = 0.5 stays that of an unstretched layout."""
    n = 4000
    lab = (np.arange(n) % 5).astype(np.int32)
    Y = synth.spread_layout(lab, scale=10.0, seed=4).astype(np.float32)
    Y[:4] = [[4000.0, 0.0], [-3000.0, 10.0], [0.0, 3500.0], [20.0, -3900.0]]
    Fe, ze = _exact_rep(Y)
    F, _, Z = oracle.repulsion_tree(Y, 0.5)
    assert np.linalg.norm(F - Fe) / np.linalg.norm(Fe) < 1e-2
    assert abs(Z - ze.sum()) / ze.sum() < 5e-3


# -------------------------------------------- random-walk estimator (Eq. 6)

import os  # noqa: E402

_GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(_GOLDEN, "splitmix64_seed1234567.txt")) if l.strip()[:1].isdigit()]
    assert [oracle.splitmix64(1234567, k) for k in range(1, 6)] == vals


def _transition_matrix(n, rp, col, X):
    """T[u, v] = exp(-|x_u - x_v|^2) / sum over N(u); a node without
    neighbours stays (T[u, u] = 1)."""
    T = np.zeros((n, n))
    for u in range(n):
        nb = col[rp[u]:rp[u + 1]]
        if nb.size == 0:
            T[u, u] = 1.0
            continue
        d2 = ((X[nb] - X[u]) ** 2).sum(1)
        w = np.exp(-(d2 - d2.min()))
        T[u, nb] = w / w.sum()
    return T


@pytest.mark.parametrize("L", [1, 2, 3])
def test_random_walk_counts_follow_the_markov_chain(L):
    """Walk counts / R estimate the L-step transition probabilities (T^L) of
    the chain with T from exp(-||x_u - x_v||^2): each count within 5 binomial
    standard deviations, and the self-returns dropped."""
    n, R = 12, 20000
    g = synth.random_graph(n, 3.0, seed=5)
    rp, col = oracle.structure(n, g.row_ptr, g.col)
    X = synth.normal(9, synth.S_MISC, 0, n * 3).reshape(n, 3) * 0.7
    wrp, wcol, wcnt = oracle.random_walk_counts(n, rp, col, X, R, L, seed=11)
    TL = np.linalg.matrix_power(_transition_matrix(n, rp, col, X), L)
    for i in range(n):
        got = np.zeros(n)
        got[wcol[wrp[i]:wrp[i + 1]]] = wcnt[wrp[i]:wrp[i + 1]]
        assert got[i] == 0
        for j in range(n):
            if j == i:
                continue
            p = TL[i, j]
            sd = np.sqrt(R * p * (1 - p)) + 1e-9
            assert abs(got[j] - R * p) <= 5 * sd + 1, (i, j, got[j], R * p)


def test_random_walk_deterministic_cases():
    # path 0-1-2-3, L = 1: the ends have one neighbour each
    n = 4
    rp, col = synth.csr_from_edges(n, np.arange(3), np.arange(1, 4))
    X = np.zeros((n, 2))
    wrp, wcol, wcnt = oracle.random_walk_counts(n, rp, col, X, 64, 1, seed=3)
    assert wcol[wrp[0]:wrp[1]].tolist() == [1] and wcnt[wrp[0]:wrp[1]].tolist() == [64]
    assert wcol[wrp[3]:wrp[4]].tolist() == [2] and wcnt[wrp[3]:wrp[4]].tolist() == [64]
    # L = 2 from an end: every walk goes 0 -> 1 -> {0, 2}; returns to 0 are dropped
    wrp, wcol, wcnt = oracle.random_walk_counts(n, rp, col, X, 64, 2, seed=3)
    assert wcol[wrp[0]:wrp[1]].tolist() == [2] and 0 < wcnt[wrp[0]] < 64
    # an isolated node keeps its walks at home: no pairs
    rp1 = np.zeros(4, np.int64)
    wrp, wcol, wcnt = oracle.random_walk_counts(3, rp1, np.zeros(0, np.int32), np.zeros((3, 2)), 8, 3)
    assert wrp.tolist() == [0, 0, 0, 0]
    # seeds: same seed same counts, another seed other counts
    g = synth.random_graph(50, 4.0, seed=1)
    r2, c2 = oracle.structure(50, g.row_ptr, g.col)
    X = synth.normal(2, synth.S_MISC, 0, 100).reshape(50, 2)
    a = oracle.random_walk_counts(50, r2, c2, X, 16, 3, seed=1)
    b = oracle.random_walk_counts(50, r2, c2, X, 16, 3, seed=1)
    c = oracle.random_walk_counts(50, r2, c2, X, 16, 3, seed=2)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not (np.array_equal(a[1], c[1]) and np.array_equal(a[2], c[2]))


def test_random_walk_P_is_a_symmetric_distribution():
    n = 300
    g = synth.random_graph(n, 5.0, seed=8)
    X = synth.block_embedding((np.arange(n) % 3).astype(np.int32), 8, seed=8) * 0.3
    rp, col, P = oracle.random_walk_P(n, g.row_ptr, g.col, X, 32, 2, seed=4)
    assert P.sum() == pytest.approx(1.0, rel=1e-12)
    assert np.all(P > 0)
    t = oracle.transpose_slots(n, rp, col)
    assert np.allclose(P, P[t], rtol=0, atol=0)


def test_gradient_rows_equal_full_gradient():
    g = synth.random_graph(400, 5.0, seed=12)
    X = synth.block_embedding((np.arange(400) % 4).astype(np.int32), 8, seed=12)
    rp, col, P = oracle.build_P(400, g.row_ptr, g.col, X, 5.0)
    Y = synth.spread_layout((np.arange(400) % 4).astype(np.int32), scale=8.0, seed=12)
    G, Z = oracle.gradient(400, rp, col, P, Y.astype(np.float64), 3.0)
    rows = np.array([0, 5, 399, 200, 17], np.int32)
    Gr = oracle.gradient_rows(400, rp, col, P, Y, 3.0, Z, rows)
    assert np.abs(Gr - G[rows]).max() <= 1e-13 * np.abs(G).max()
    # Z from the row sums of repulsion_all equals the full Z
    _, zr = oracle.repulsion_all(Y, threads=3)
    assert zr.sum() == pytest.approx(Z, rel=1e-13)

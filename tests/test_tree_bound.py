"""The oracle's tree code against the EXACT repulsive sums (Eq. 4), under the
error bound derived for the monopole approximation.

The tree code replaces the m exact terms of an accepted node by m copies of
one term at the node's centre of mass.  Taylor's theorem with the integral
remainder bounds, for every row i and every node accepted for i, the
difference by the node's centre rounding (first order) plus
1/2 sum_j |c - y_j|^2 times the largest second derivative of w, or of w^2 u,
at distance >= |y_i - c| - a from the origin (a: the farthest box corner
from c); the derivation sits above ``node_bound`` in the oracle's C source.
``oracle.repulsion_tree_bounds`` returns that bound per row, summed over the
accepted nodes, and these tests check every row of the tree code against
the plain O(n^2) rows of ``oracle.repulsion_all`` under it.

None of this reuses the tree code's arithmetic as the reference: the
reference is the exact definition, and the bound is a property of the
approximation, so a mistake in the tree code (a wrong count, centre or
sign, a self-pair) shows up as a row outside its bound, or, for a centre
shifted to first order, as a departure from a closed form
(``test_planted_mistakes_are_caught``).
"""

import numpy as np
import pytest

import oracle
import tsgne_synth as synth


def _layout(kind, n, seed):
    labels = (np.arange(n) % 7).astype(np.int32)
    if kind == "spread":
        Y = synth.spread_layout(labels, scale=20.0, seed=seed)
    elif kind == "tiny":
        Y = synth.y_init(n, sigma=1e-4, seed=seed)
    elif kind == "outliers":
        Y = synth.spread_layout(labels, scale=5.0, seed=seed)
        Y[:5] *= 400.0  # a few points 400x farther out than the bulk
    elif kind == "coincident":
        Y = synth.spread_layout(labels, scale=5.0, seed=seed)
        Y[: n // 3] = Y[0]  # a third of the points on one spot
    elif kind == "clusters":
        rng = np.random.default_rng(seed)
        Y = np.concatenate([rng.normal(size=(n // 2, 2)) * 0.3,
                            rng.normal(size=(n - n // 2, 2)) * 0.3 + [60.0, -20.0]])
    else:
        raise ValueError(kind)
    return np.asarray(Y, np.float32).astype(np.float64)  # FP32 values, as the tree code reads them


def _abs_force_sums(Y):
    """A_i = sum_{j != i} |w_ij^2 (y_i - y_j)| (a scale for rounding slack)."""
    n = Y.shape[0]
    A = np.zeros(n)
    for a in range(0, n, 512):
        d = Y[a:a + 512, None, :] - Y[None, :, :]
        r2 = (d * d).sum(-1)
        w = 1.0 / (1.0 + r2)
        A[a:a + 512] = (w * w * np.sqrt(r2)).sum(1)
    return A


def _check_rows(Y, theta):
    """(F, zr, Z, bZ, bF, Fe, zre, A) with every row checked against the bound."""
    F, zr, Z, bZ, bF = oracle.repulsion_tree_bounds(Y, theta)
    Fe, zre = oracle.repulsion_all(Y)
    A = _abs_force_sums(Y)
    eF = np.linalg.norm(F - Fe, axis=1)
    eZ = np.abs(zr - zre)
    BF = bF.sum(1)
    BZ = bZ.sum(1)
    # FP64 rounding of two sums of up to n terms of each row
    slackF = 1e-12 * A + 1e-300
    slackZ = 1e-12 * zre
    return F, zr, Z, bZ, bF, Fe, zre, A, eF, eZ, BF, BZ, slackF, slackZ


CASES = [(n, kind, th) for n, kind in [(2000, "spread"), (5003, "outliers"), (5003, "tiny"), (9000, "coincident"),
                                         (3000, "clusters")]
         for th in (0.3, 0.5, 0.8, 1.0)]


@pytest.mark.parametrize("n,kind,theta", CASES)
def test_tree_code_stays_within_the_derived_bound(n, kind, theta):
    Y = _layout(kind, n, seed=n)
    F, zr, Z, bZ, bF, Fe, zre, A, eF, eZ, BF, BZ, slackF, slackZ = _check_rows(Y, theta)
    bad = np.flatnonzero(eF > BF + slackF)
    assert bad.size == 0, (bad[:5], eF[bad[:5]], BF[bad[:5]])
    bad = np.flatnonzero(eZ > BZ + slackZ)
    assert bad.size == 0, (bad[:5], eZ[bad[:5]], BZ[bad[:5]])
    Ze = float(zre.sum())
    assert abs(Z - Ze) <= BZ.sum() + 1e-12 * Ze
    # the first-order part is the FP32 rounding of the centres only: a wrong
    # centre would put it far above this
    assert (bF[:, 0] <= 1e-4 * A + 1e-300).all()
    assert (bZ[:, 0] <= 1e-4 * zre).all()


@pytest.mark.parametrize("theta", [0.3, 0.5])
def test_the_bound_is_informative_on_a_spread_layout(theta):
    """Rows' bounds are a small fraction of their absolute force sums and
    within a factor of a few tens of the actual error of the worst row."""
    Y = _layout("spread", 5003, seed=3)
    F, zr, Z, bZ, bF, Fe, zre, A, eF, eZ, BF, BZ, slackF, slackZ = _check_rows(Y, theta)
    assert np.median(BF / A) < (0.1 if theta == 0.3 else 0.3)
    assert BZ.sum() / zre.sum() < (0.015 if theta == 0.3 else 0.05)
    assert (eF / np.maximum(BF, 1e-300)).max() > 0.005  # not a vacuous bound


def test_theta_zero_has_a_zero_bound_and_equals_the_exact_rows():
    Y = _layout("spread", 1500, seed=5)
    F, zr, Z, bZ, bF = oracle.repulsion_tree_bounds(Y, 0.0)
    Fe, zre = oracle.repulsion_all(Y)
    assert (bZ == 0).all() and (bF == 0).all()
    assert np.abs(F - Fe).max() <= 1e-12 * np.abs(Fe).max()
    assert np.abs(zr - zre).max() <= 1e-12 * zre.max()


def _lopsided_far_clusters_match_monopoles(Y, F, zr):
    """Closed form: two 32-point clusters 100 apart see each other as one
    node of weight 32 at the other cluster's mean; within a cluster every
    pair is exact.  The clusters are lopsided (most points in one corner),
    so the mean is far from the box centre."""
    for own, other in ((slice(0, 32), slice(32, 64)), (slice(32, 64), slice(0, 32))):
        c = Y[other].mean(0)
        for i in range(own.start, own.stop):
            e = Y[i] - Y[own]
            w = 1.0 / (1.0 + (e ** 2).sum(1))
            m = np.arange(own.start, own.stop) != i
            wc = 1.0 / (1.0 + ((Y[i] - c) ** 2).sum())
            f = ((w[m] ** 2)[:, None] * e[m]).sum(0) + 32 * wc ** 2 * (Y[i] - c)
            z = w[m].sum() + 32 * wc
            if not (np.allclose(F[i], f, rtol=1e-9, atol=0) and abs(zr[i] - z) <= 1e-9 * z):
                return False
    return True


def _lopsided_clusters():
    rng = np.random.default_rng(11)
    A = rng.uniform(0, 1, size=(32, 2)) ** 4 - 0.5  # bunched near (-0.5, -0.5)
    B = rng.uniform(0, 1, size=(32, 2)) ** 4 - 0.5 + [100.0, 0.0]
    return np.concatenate([A, B]).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(mutation):
    """Each planted mistake in the tree code (1: count one short, 3: force
    sign, 4: a self pair in an exact bucket) puts rows outside the derived
    bound; 2 (the box centre in place of the centre of mass) is a
    first-order shift that the second-order bound can hide, so it is
    caught by the closed form of two lopsided far clusters instead."""
    Yc = _lopsided_clusters()
    Y = _layout("spread", 3000, seed=9)
    try:
        oracle.tree_mutation(mutation)
        if mutation == 2:
            F, zr, _ = oracle.repulsion_tree(Yc, 0.5)
            caught = not _lopsided_far_clusters_match_monopoles(Yc, F, zr)
        else:
            F, zr, Z, bZ, bF, Fe, zre, A, eF, eZ, BF, BZ, slackF, slackZ = _check_rows(Y, 0.3)
            caught = (eF > BF + slackF).sum() + (eZ > BZ + slackZ).sum() > 0
    finally:
        oracle.tree_mutation(0)
    assert caught, mutation
    # the unmutated code passes both checks
    F, zr, _ = oracle.repulsion_tree(Yc, 0.5)
    assert _lopsided_far_clusters_match_monopoles(Yc, F, zr)
    F, zr, Z, bZ, bF, Fe, zre, A, eF, eZ, BF, BZ, slackF, slackZ = _check_rows(Y, 0.3)
    assert ((eF <= BF + slackF).all() and (eZ <= BZ + slackZ).all())


def test_hessian_bounds_against_sampled_second_differences():
    """The closed-form sup of the second directional derivatives used by the
    bound dominates central second differences of w and w^2 u sampled over
    radii and directions (checks the derivatives, independently of any
    tree)."""
    rng = np.random.default_rng(0)

    def w(x):
        return 1.0 / (1.0 + (x * x).sum(-1))

    def f(x):
        return (w(x) ** 2)[..., None] * x

    def G_w(rho):
        s = rho * rho
        ww = 1.0 / (1.0 + s)
        return np.where(s <= 1.0, 2 * ww * ww, 2 * ww ** 3 * (3 * s - 1))

    def G_f(rho):
        t = np.maximum(rho, 1 / np.sqrt(3.0))
        return (12 * t + 36 * t ** 3) / (1 + t * t) ** 4

    h = 1e-4
    for _ in range(2000):
        r = rng.uniform(0, 6)
        phi, psi = rng.uniform(0, 2 * np.pi, 2)
        x = r * np.array([np.cos(phi), np.sin(phi)])
        d = np.array([np.cos(psi), np.sin(psi)])
        d2w = (w(x + h * d) - 2 * w(x) + w(x - h * d)) / h ** 2
        d2f = (f(x + h * d) - 2 * f(x) + f(x - h * d)) / h ** 2
        assert abs(d2w) <= G_w(r) * (1 + 1e-5) + 1e-6
        assert np.linalg.norm(d2f) <= G_f(r) * (1 + 1e-5) + 1e-6

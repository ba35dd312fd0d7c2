"""The paper's two layout-quality measures, computed on the host from a
finished layout (reporting only; not part of the GPU iteration).

NMI (Sec. 2.5, Eq. 11): NMI(PR; TR) = 2 I(PR; TR) / (H(PR) + H(TR)) between
the graph's communities and a clustering of the 2-D layout with the same
number of clusters.  Readings: the paper's "kNN clustering" of the layout is
read as k-means (Lloyd's iterations from k-means++ seeds, best of a few seeded
restarts); the graph communities are the planted blocks of the synthetic
graphs (the paper uses Louvain on real graphs).  Higher is more similar, as
the definition and the paper's tables imply.

AQ (Sec. 2.6, Eqs. 12-14): a k x k grid over the bounding box of the layout;
a cell is good when one community's share of its points is larger than p;
AQ = good cells / k^2.  The paper gives neither k nor p; the defaults are
k = 10 and p = 0.5, empty cells are not good, and points on the maximum edge
fall in the last cell.
"""

from __future__ import annotations

import numpy as np

__all__ = ["nmi", "aq", "kmeans", "layout_nmi"]


def _entropy(counts: np.ndarray) -> float:
    p = counts[counts > 0] / counts.sum()
    return float(-(p * np.log(p)).sum())


def nmi(a, b) -> float:
    """2 I(a; b) / (H(a) + H(b)) of two labelings (Eq. 11)."""
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    joint = np.zeros((ai.max() + 1, bi.max() + 1))
    np.add.at(joint, (ai, bi), 1.0)
    ha = _entropy(joint.sum(1))
    hb = _entropy(joint.sum(0))
    if ha + hb == 0.0:
        return 1.0
    pj = joint / joint.sum()
    pa = pj.sum(1, keepdims=True)
    pb = pj.sum(0, keepdims=True)
    m = pj > 0
    mi = float((pj[m] * np.log(pj[m] / (pa @ pb)[m])).sum())
    return 2.0 * mi / (ha + hb)


def kmeans(Y, k: int, restarts: int = 3, iters: int = 50, seed: int = 0):
    """Lloyd's k-means with k-means++ seeding; returns (labels, inertia) of the best restart."""
    Y = np.asarray(Y, np.float64)
    n = Y.shape[0]
    rng = np.random.default_rng(seed)
    best = (None, np.inf)
    y2 = (Y * Y).sum(1)
    for _ in range(restarts):
        c = np.empty((k, Y.shape[1]))
        c[0] = Y[rng.integers(n)]
        d2 = ((Y - c[0]) ** 2).sum(1)
        for t in range(1, k):
            pr = d2 / d2.sum() if d2.sum() > 0 else np.full(n, 1.0 / n)
            c[t] = Y[rng.choice(n, p=pr)]
            d2 = np.minimum(d2, ((Y - c[t]) ** 2).sum(1))
        lab = None
        for _ in range(iters):
            dist = y2[:, None] - 2.0 * Y @ c.T + (c * c).sum(1)[None, :]
            new = dist.argmin(1)
            if lab is not None and np.array_equal(new, lab):
                break
            lab = new
            for t in range(k):
                m = lab == t
                if m.any():
                    c[t] = Y[m].mean(0)
        inertia = float(((Y - c[lab]) ** 2).sum())
        if inertia < best[1]:
            best = (lab.copy(), inertia)
    return best


def layout_nmi(Y, communities, restarts: int = 3, seed: int = 0) -> float:
    """NMI between the communities and a k-means clustering of Y with k = #communities."""
    communities = np.asarray(communities)
    k = int(np.unique(communities).size)
    lab, _ = kmeans(Y, k, restarts=restarts, seed=seed)
    return nmi(communities, lab)


def aq(Y, communities, k: int = 10, p: float = 0.5) -> float:
    """Aesthetic quality (Eqs. 12-14): share of grid cells dominated (> p) by one community."""
    Y = np.asarray(Y, np.float64)
    communities = np.asarray(communities)
    lo = Y.min(0)
    hi = Y.max(0)
    span = np.where(hi > lo, hi - lo, 1.0)
    cell = np.minimum(((Y - lo) / span * k).astype(np.int64), k - 1)
    idx = cell[:, 0] * k + cell[:, 1]
    _, ci = np.unique(communities, return_inverse=True)
    counts = np.zeros((k * k, ci.max() + 1))
    np.add.at(counts, (idx, ci), 1.0)
    tot = counts.sum(1)
    good = (tot > 0) & (counts.max(1) > p * np.maximum(tot, 1))
    return float(good.sum()) / float(k * k)

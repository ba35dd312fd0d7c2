"""Pins for the host-side quality measures NMI (Eq. 11) and AQ (Eqs. 12-14)."""

import math

import numpy as np
import pytest

from paper_2310_11186_gb300 import quality


def test_nmi_identical_and_relabelled():
    a = np.array([0, 0, 1, 1, 2, 2, 2])
    assert quality.nmi(a, a) == pytest.approx(1.0)
    assert quality.nmi(a, (a + 5) * 3) == pytest.approx(1.0)  # labels are names only


def test_nmi_independent_is_near_zero():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 5, 200000)
    b = rng.integers(0, 7, 200000)
    assert quality.nmi(a, b) < 1e-3


def test_nmi_hand_example():
    """a = (0,0,1,1), b = (0,1,1,1): H(a) = ln 2, H(b) = -(1/4 ln 1/4 + 3/4 ln 3/4),
    I = H(b) - H(b|a) = H(b) - 1/2 ln 2."""
    a = [0, 0, 1, 1]
    b = [0, 1, 1, 1]
    ha = math.log(2)
    hb = -(0.25 * math.log(0.25) + 0.75 * math.log(0.75))
    want = 2 * (hb - 0.5 * math.log(2)) / (ha + hb)
    assert quality.nmi(a, b) == pytest.approx(want, rel=1e-12)


def test_aq_two_separated_clusters():
    """Two clusters in opposite corners of the bounding box: exactly the two
    corner cells hold points and both are pure -> AQ = 2 / k^2."""
    Y = np.array([[0.0, 0.0], [0.05, 0.02], [1.0, 1.0], [0.97, 0.99]])
    c = np.array([0, 0, 1, 1])
    assert quality.aq(Y, c, k=10, p=0.5) == pytest.approx(2 / 100)
    # a mixed cell with an even split is not good (share must exceed p)
    Y2 = np.array([[0.0, 0.0], [0.01, 0.0], [1.0, 1.0]])
    c2 = np.array([0, 1, 1])
    assert quality.aq(Y2, c2, k=2, p=0.5) == pytest.approx(1 / 4)


def test_kmeans_recovers_separated_blobs():
    rng = np.random.default_rng(1)
    centres = np.array([[0, 0], [20, 0], [0, 20], [20, 20]], float)
    lab = np.repeat(np.arange(4), 250)
    Y = centres[lab] + rng.normal(size=(1000, 2))
    assert quality.layout_nmi(Y, lab) == pytest.approx(1.0)

"""Pins of the oracle's solid ratio (Sec. 2.3, Fig. 3) against brute force.

The exact disk-cell overlap is checked against 1000 x 1000 sub-sampling of the
cell (the area as a count), against the disk area pi r^2 summed over all cells,
and against its limits; the cell decomposition of Fig. 3b (n_sub sub-cells) is
checked to converge to the exact area.
"""
import math

import numpy as np
import pytest


def _brute_area(a0, b0, r, n=1000):
    # midpoint sampling of the unit cell [a0, a0+1] x [b0, b0+1] (disk centred at the origin)
    t = (np.arange(n) + 0.5) / n
    X = a0 + t[None, :]
    Y = b0 + t[:, None]
    return np.count_nonzero(X * X + Y * Y <= r * r) / (n * n)


@pytest.mark.parametrize("r", [1.3, 3.7, 8.0, 10.0, 12.0])
def test_exact_area_matches_subsampling(orc, r):
    rng = np.random.default_rng(int(r * 10))
    worst = 0.0
    tested = 0
    for _ in range(400):
        ang = rng.uniform(0, 2 * math.pi)
        rad = r + rng.uniform(-1.5, 1.5)
        a0 = math.floor(rad * math.cos(ang)) + rng.uniform(-0.5, 0.5)
        b0 = math.floor(rad * math.sin(ang)) + rng.uniform(-0.5, 0.5)
        exact = orc.cell_area(a0, a0 + 1, b0, b0 + 1, r)
        if 0.0 < exact < 1.0:
            tested += 1
        worst = max(worst, abs(exact - _brute_area(a0, b0, r)))
        if tested >= 40:
            break
    assert tested >= 20
    assert worst < 1e-4


@pytest.mark.parametrize("cx,cy,r", [(0.3, 0.7, 10.0), (0.5, 0.5, 8.0), (0.01, 0.99, 12.0),
                                     (0.25, 0.0, 3.0), (0.77, 0.13, 1.1)])
def test_exact_area_sums_to_disk_area(orc, cx, cy, r):
    # sum over all cells of the overlap = pi r^2 (partition of the plane)
    tot = 0.0
    span = int(math.ceil(r)) + 2
    for k in range(-span, span + 1):
        for i in range(-span, span + 1):
            tot += orc.cell_area(i - cx, i + 1 - cx, k - cy, k + 1 - cy, r)
    assert abs(tot - math.pi * r * r) < 1e-12 * r * r


def test_exact_area_limits(orc):
    assert orc.cell_area(20.0, 21.0, 0.0, 1.0, 10.0) == 0.0        # far outside
    assert orc.cell_area(-0.5, 0.5, -0.5, 0.5, 10.0) == pytest.approx(1.0, abs=1e-14)   # deep inside
    assert orc.cell_area(6.0, 7.0, 6.0, 7.0, 10.0) == pytest.approx(1.0, abs=1e-14)    # corner at 9.9
    # a cell that only touches the circle at its nearest corner has no overlap
    assert orc.cell_area(10.0, 11.0, 0.0, 1.0, 10.0) == 0.0


def test_exact_area_symmetries(orc):
    rng = np.random.default_rng(11)
    for _ in range(50):
        a0, b0 = rng.uniform(-11, 10, 2)
        r = rng.uniform(2, 12)
        v = orc.cell_area(a0, a0 + 1, b0, b0 + 1, r)
        assert orc.cell_area(-a0 - 1, -a0, b0, b0 + 1, r) == pytest.approx(v, abs=1e-12)
        assert orc.cell_area(b0, b0 + 1, a0, a0 + 1, r) == pytest.approx(v, abs=1e-12)


def test_half_disk_and_quarter_cell(orc):
    # a straight line through the centre halves the overlap of a centred unit cell
    assert orc.cell_area(-0.5, 0.5, -0.5, 0.0, 10.0) == pytest.approx(0.5, abs=1e-14)
    # quarter disk in a box: r = 0.9 inside [0, 1]^2 -> pi r^2 / 4
    assert orc.cell_area(0.0, 1.0, 0.0, 1.0, 0.9) == pytest.approx(math.pi * 0.81 / 4, abs=1e-14)


@pytest.mark.parametrize("n,expect", [(2, 2 / 4), (5, 11 / 25), (10, 50 / 100)])
def test_subcell_decomposition_counts(orc, n, expect):
    # Fig. 3b worked by hand: the unit cell [-100.5, -99.5] x [-0.5, 0.5] straddles the left
    # edge x = -100 of a disk of radius 100 centred at the origin.  Sub-cell centres right of
    # x = -100 are inside (the boundary bulges out by at most 0.5^2/200 < 1/(2n)); for odd n
    # the centre (-100, 0) lies exactly on the circle and a tie counts as inside:
    # n = 2 -> 1 column x 2 rows; n = 5 -> 2 columns x 5 rows + 1 tie; n = 10 -> 5 x 10.
    assert orc.eps_subcell(-100.5, -0.5, 100.0, n) == expect


def test_subcell_converges_to_exact(orc):
    rng = np.random.default_rng(12)
    for _ in range(20):
        r = rng.uniform(4, 12)
        ang = rng.uniform(0, 2 * math.pi)
        a0 = math.floor(r * math.cos(ang)) + 0.0
        b0 = math.floor(r * math.sin(ang)) + 0.0
        ex = orc.cell_area(a0, a0 + 1, b0, b0 + 1, r)
        e5 = orc.eps_subcell(a0, b0, r, 5)
        e200 = orc.eps_subcell(a0, b0, r, 200)
        assert abs(e200 - ex) < 5e-3
        assert abs(e5 - ex) < 0.25


def test_coverage_decision_matches_positive_area(orc):
    # a cell is listed for a disk iff the disk reaches into it: away from tangency the
    # single-precision nearest-point test agrees with a positive exact overlap
    rng = np.random.default_rng(13)
    for _ in range(2000):
        r = rng.uniform(2, 12)
        a0, b0 = rng.uniform(-r - 2, r + 1, 2)
        ex = orc.cell_area(a0, a0 + 1, b0, b0 + 1, r)
        dx = a0 if a0 > 0 else (a0 + 1 if a0 + 1 < 0 else 0.0)
        dy = b0 if b0 > 0 else (b0 + 1 if b0 + 1 < 0 else 0.0)
        if abs(math.hypot(dx, dy) - r) < 1e-4:
            continue
        assert orc.covers(a0, b0, r) == (ex > 0.0)

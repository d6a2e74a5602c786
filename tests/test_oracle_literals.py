"""Pins of the oracle's covariance, knot grid and partition to literal values.

The recursion pins (test_oracle_pins.py) compare the oracle with checkers that
share its tree; these tests fix the pieces that tree is made of against values
worked out by hand from the paper's definitions, so that a slip in any of them
(a dropped sqrt(3) in Eq. mat15, a distance not divided by the range, knots on
the region boundary, a midpoint sent to the lower child) turns a test red.
The literals are the closed forms named beside each, evaluated to 20 digits.
"""
import math

import numpy as np
import pytest

from oracle import exact as E
from oracle import mra_oracle as O

# e^{-h} and (1 + sqrt3 h) e^{-sqrt3 h} (Eq. mat15) at h = 1/2, 1, 2
EXP = {0.5: 0.6065306597126334236, 1.0: 0.3678794411714423216, 2.0: 0.13533528323661269189}
M15 = {0.5: 0.78488765395745065448, 1.0: 0.4833577245965076506, 2.0: 0.13973135019231467094}


@pytest.mark.parametrize("family,table", [("exp", EXP), ("matern15", M15)])
@pytest.mark.parametrize("impl", ["oracle", "checker"])
def test_cov_literal_values(family, table, impl):
    """C0 at h = 0, kappa/2, kappa, 2 kappa along both axes (Sec. 2.1, Eq. mat15, Sec. 4.2)."""
    f = O.cov if impl == "oracle" else E.c0
    sigma2, kappa = 1.7, 0.2
    s0 = np.array([[0.3, 0.6]])
    for frac, rho in table.items():
        for axis in (0, 1):
            s1 = s0.copy()
            s1[0, axis] += frac * kappa
            got = f(s0, s1, (sigma2, kappa), family)[0, 0]
            assert got == pytest.approx(sigma2 * rho, rel=1e-14)
    assert f(s0, s0, (sigma2, kappa), family)[0, 0] == pytest.approx(sigma2, rel=1e-15)
    # a diagonal offset of length kappa: (0.6 kappa, 0.8 kappa)
    s1 = s0 + np.array([[0.6 * kappa, 0.8 * kappa]])
    assert f(s0, s1, (sigma2, kappa), family)[0, 0] == pytest.approx(sigma2 * table[1.0], rel=1e-14)


@pytest.mark.parametrize("impl", ["oracle", "checker"])
def test_cov_nonstationary_literals(impl):
    """Variance sigma2 sqrt(g(s1) g(s2)), g(s) = 1 + sin(4 pi s_x)/2 (reading R12):
    g(0) = 1, g(1/8) = 3/2, g(1/4) = 1."""
    f = O.cov if impl == "oracle" else E.c0
    pts = np.array([[0.0, 0.5], [0.125, 0.5], [0.25, 0.5]])
    C = f(pts, pts, (2.0, 0.25), "exp", nonstat=True)
    assert np.diag(C) == pytest.approx([2.0, 3.0, 2.0], rel=1e-14)
    # distance 1/8 = kappa / 2: 2 sqrt(3/2) e^{-1/2}
    assert C[0, 1] == pytest.approx(1.4856906296496097675, rel=1e-14)
    assert C[1, 2] == pytest.approx(1.4856906296496097675, rel=1e-14)
    # distance 1/4 = kappa, g = 1 at both ends: 2 e^{-1}
    assert C[0, 2] == pytest.approx(2.0 * EXP[1.0], rel=1e-14)
    C15 = f(pts[:2], pts[:2], (2.0, 0.25), "matern15", nonstat=True)
    # 2 sqrt(3/2) (1 + sqrt3/2) e^{-sqrt3/2}
    assert C15[0, 1] == pytest.approx(1.9225742576059279027, rel=1e-14)


def test_general_matern_reduces_to_closed_forms():
    """The checker's Bessel-function Matern equals the half-integer closed forms
    (nu = 1/2: e^{-h}; nu = 3/2: Eq. mat15; nu = 5/2: (1 + sqrt5 h + 5 h^2/3) e^{-sqrt5 h})."""
    h = np.linspace(0.0, 4.0, 41)
    np.testing.assert_allclose(E.matern(h, 0.5), np.exp(-h), rtol=1e-13)
    np.testing.assert_allclose(E.matern(h, 1.5), (1 + math.sqrt(3) * h) * np.exp(-math.sqrt(3) * h), rtol=1e-13)
    s5 = math.sqrt(5.0)
    np.testing.assert_allclose(E.matern(h, 2.5), (1 + s5 * h + 5 * h * h / 3) * np.exp(-s5 * h), rtol=1e-13)


# Reading R8: cell-centred g_x x g_y grid, x fastest; g_x = smallest divisor of r with g_x^2 >= r.
CENTRES4 = [0.125, 0.375, 0.625, 0.875]
CENTRES8 = [0.0625, 0.1875, 0.3125, 0.4375, 0.5625, 0.6875, 0.8125, 0.9375]


@pytest.mark.parametrize("r,xs,ys", [(16, CENTRES4, CENTRES4), (32, CENTRES8, CENTRES4), (64, CENTRES8, CENTRES8),
                                     (4, [0.25, 0.75], [0.25, 0.75]), (2, [0.25, 0.75], [0.5])])
def test_grid_knots_literal(r, xs, ys):
    k = O.grid_knots((0.0, 1.0, 0.0, 1.0), r, 2)
    want = np.array([[x, y] for y in ys for x in xs])
    assert k.shape == (r, 2)
    np.testing.assert_array_equal(k, want)


def test_grid_knots_of_a_subregion():
    """Region [1/2, 1] x [1/4, 1/2] (level-2 child 3 of child 1) with r = 4."""
    k = O.grid_knots((0.5, 1.0, 0.25, 0.5), 4, 2)
    np.testing.assert_array_equal(k, [[0.625, 0.3125], [0.875, 0.3125], [0.625, 0.4375], [0.875, 0.4375]])


def test_grid_knots_never_on_coarser_knots():
    """Nested cell-centred grids never coincide across levels (reading R8)."""
    t = O.build_tree(np.array([[0.1, 0.1]]), M=3, r=16)
    coarse = {tuple(q) for m in range(2) for b in t.knots[m] for q in b}
    fine = {tuple(q) for b in t.knots[2] for q in b}
    assert not coarse & fine


# Reading R9: half-open midpoint split, child j = b_x + 2 b_y, last cell closed.
PTS = [((0.0, 0.0), 0, 0), ((0.5, 0.5), 3, 12), ((0.5, 0.25), 1, 6), ((0.25, 0.5), 2, 9),
       ((0.75, 0.25), 1, 7), ((1.0, 1.0), 3, 15), ((1.0, 0.0), 1, 5), ((0.0, 1.0), 2, 10),
       ((0.49, 0.74), 2, 9), ((0.25, 0.25), 0, 3)]


@pytest.mark.parametrize("impl", ["oracle", "checker"])
def test_partition_literal_leaves(impl):
    pts = np.array([p for p, _, _ in PTS])
    for M, col in ((1, 1), (2, 2)):
        want = [w[col] for w in PTS]
        if impl == "oracle":
            got = O.locate(pts, O.build_tree(pts, M=M, r=4).boxes, 4, M, 2)
        else:
            got = E.cell_index(pts, (0.0, 1.0, 0.0, 1.0), 4, M, 2)
        np.testing.assert_array_equal(got, want)


def test_build_tree_leaf_lists_and_boxes():
    pts = np.array([p for p, _, _ in PTS])
    t = O.build_tree(pts, M=2, r=4)
    assert t.boxes[1][1] == (0.5, 1.0, 0.0, 0.5)
    assert t.boxes[2][7] == (0.75, 1.0, 0.25, 0.5)
    for k, (_, _, leaf) in enumerate(PTS):
        assert k in t.obs[leaf]
    assert sum(len(o) for o in t.obs) == len(PTS)
    # stable: original order inside a leaf
    t2 = O.build_tree(np.array([[0.9, 0.9], [0.8, 0.8], [0.95, 0.99]]), M=1, r=4)
    np.testing.assert_array_equal(t2.obs[3], [0, 1, 2])


@pytest.mark.parametrize("nu,table", [(0.5, EXP), (1.5, M15)])
def test_free_smoothness_family_at_half_integers(nu, table):
    """The family "matern" (Sec. 4.1) equals the closed forms at nu = 1/2 and 3/2."""
    sigma2, kappa = 0.9, 0.3
    s0 = np.array([[0.2, 0.1]])
    for frac, rho in table.items():
        s1 = s0 + np.array([[0.0, frac * kappa]])
        assert O.cov(s0, s1, (sigma2, kappa, nu), "matern")[0, 0] == pytest.approx(sigma2 * rho, rel=1e-13)
    assert O.cov(s0, s0, (sigma2, kappa, 2.7), "matern")[0, 0] == pytest.approx(sigma2, rel=1e-15)


# Reading R18: level-varying J (Sec. 2.2; Sec. 4.3's (2, 2, 4, 8, 8, 16)).  Each
# level's log2 J_m midpoint halvings go to the axis halved fewer times so far
# (x on ties); child j = c_x + s_x c_y.  Values worked by hand.
def test_level_varying_J_halvings():
    assert [O.halvings((2, 2, 4, 8, 8, 16), m) for m in range(1, 7)] == \
        [(1, 0), (0, 1), (1, 1), (2, 1), (1, 2), (2, 2)]          # 128 x 128 square leaves
    assert [O.halvings(4, m) for m in range(1, 4)] == [(1, 1)] * 3   # the quadtree
    with pytest.raises(ValueError):
        O.halvings((2, 6), 2)


def test_level_varying_J_boxes():
    t = O.build_tree(np.array([[0.1, 0.1]]), M=2, J=(2, 8), r=4)
    assert t.boxes[1] == [(0.0, 0.5, 0.0, 1.0), (0.5, 1.0, 0.0, 1.0)]
    want = {0: (0.0, 0.25, 0.0, 0.25), 1: (0.25, 0.5, 0.0, 0.25), 2: (0.0, 0.25, 0.25, 0.5),
            7: (0.25, 0.5, 0.75, 1.0), 8: (0.5, 0.75, 0.0, 0.25), 15: (0.75, 1.0, 0.75, 1.0)}
    for i, b in want.items():
        assert t.boxes[2][i] == b
    assert len(t.boxes[2]) == 16 and t.nreg(2) == 16
    assert O.ancestors(2, 13, (2, 8)) == [(0, 0), (1, 1), (2, 13)]


# (point, leaf under J = (2, 8), leaf under J = (16,): the 4 x 4 grid, j = floor(4x) + 4 floor(4y))
PTS_J = [((0.5, 0.25), 10, 6), ((1.0, 1.0), 15, 15), ((0.25, 0.75), 7, 13), ((0.0, 0.0), 0, 0),
         ((0.49, 0.74), 5, 9), ((0.75, 0.5), 13, 11), ((0.1, 0.3), 2, 4)]


@pytest.mark.parametrize("impl", ["oracle", "checker"])
def test_level_varying_J_literal_leaves(impl):
    pts = np.array([p for p, _, _ in PTS_J])
    for J, col in (((2, 8), 1), ((16,), 2)):
        want = [w[col] for w in PTS_J]
        M = len(J)
        if impl == "oracle":
            got = O.locate(pts, O.build_tree(pts, M=M, J=J, r=4).boxes, J, M, 2)
        else:
            got = E.cell_index(pts, (0.0, 1.0, 0.0, 1.0), J, M, 2)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("J", [(2, 2, 4, 8), (8, 2), (16, 4), (4, 4, 4), (2, 16)])
def test_level_varying_J_locators_agree(J):
    """The oracle's descent and the checker's integer-cell locator (two
    independent statements of R18) agree at every level, on random points and on
    every cell boundary of the finest grid."""
    rng = np.random.default_rng(len(J) + sum(J))
    L = int(round(np.log2(np.prod(J))))
    gx, gy = 2 ** ((L + 1) // 2), 2 ** (L // 2)
    edge = np.array([[i / gx, j / gy] for i in range(gx + 1) for j in range(gy + 1)])
    pts = np.concatenate([rng.random((400, 2)), edge])
    t = O.build_tree(pts, M=len(J), J=J, r=4)
    for m in range(1, len(J) + 1):
        np.testing.assert_array_equal(O.locate(pts, t.boxes, J[:m], m, 2), E.cell_index(pts, (0, 1, 0, 1), J, m, 2))
    assert sum(len(o) for o in t.obs) == pts.shape[0]


@pytest.mark.parametrize("J", [(2, 8, 2), (16, 4), (2, 2, 4, 8, 8, 16)])
def test_level_varying_J_points_lie_in_their_boxes(J):
    """Every point lies in the half-open box of its region at every level (closed
    at the bounding box maximum), and the boxes of a level tile the domain: the
    partition's boxes and its point locator state the same regions."""
    rng = np.random.default_rng(sum(J))
    pts = np.concatenate([rng.random((300, 2)), [[1.0, 1.0], [0.0, 1.0], [1.0, 0.0], [0.5, 0.5]]])
    M = len(J)
    t = O.build_tree(pts, M=M, J=J, r=4)
    for m in range(1, M + 1):
        b = np.asarray(t.boxes[m])
        assert np.isclose(np.sum((b[:, 1] - b[:, 0]) * (b[:, 3] - b[:, 2])), 1.0, rtol=0, atol=1e-12)
        leaf = O.locate(pts, t.boxes, J[:m], m, 2)
        x0, x1, y0, y1 = b[leaf].T
        inx = (pts[:, 0] >= x0) & ((pts[:, 0] < x1) | (x1 == 1.0))
        iny = (pts[:, 1] >= y0) & ((pts[:, 1] < y1) | (y1 == 1.0))
        assert inx.all() and iny.all()

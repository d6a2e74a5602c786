"""Host-side partition planning (Sec. 2.2, 2.5, 4.3): no GPU.

The occupancy of the planner's cells is checked against the oracle's own
partition (the leaves of a tree built with the chosen J), so a planner whose
grid disagreed with the partition the library builds would fail here.
"""
import numpy as np
import pytest

from oracle import mra_oracle as O
from paper_1507_04789_gb300 import plan


def _grid_points(k):
    g = (np.arange(k) + 0.5) / k
    return np.stack(np.meshgrid(g, g), -1).reshape(-1, 2)


def test_choose_levels_on_a_regular_grid():
    locs = _grid_points(64)                      # 4096 points, one per cell of the 64 x 64 grid
    assert plan.choose_levels(locs, max_leaf=1) == 6
    assert plan.choose_levels(locs, max_leaf=4) == 5
    assert plan.choose_levels(locs, max_leaf=4096) == 0


@pytest.mark.parametrize("M,max_leaf,last_max,want", [
    (5, 4, 4, (4, 4, 4, 4, 4)),                  # 10 halvings: the quadtree
    (6, 4, 4, (2, 2, 4, 4, 4, 4)),               # 10 halvings over 6 levels, the remainder fine
    (6, 1, 4, (4, 4, 4, 4, 4, 4)),               # 12 halvings
    (4, 1, 16, (4, 8, 8, 16)),                   # 12 halvings, J_M up to 16: the paper's rising shape
    (3, 1, 16, (16, 16, 16)),
])
def test_choose_J_levels_literal(M, max_leaf, last_max, want):
    assert plan.choose_J_levels(_grid_points(64), M, max_leaf=max_leaf, last_max=last_max) == want


@pytest.mark.parametrize("M,last_max", [(6, 4), (7, 4), (5, 16)])
def test_choose_J_levels_bounds_the_leaves(M, last_max):
    """The chosen tree's leaves hold at most max_leaf points, and one halving
    fewer would not: checked on the oracle's partition with that J."""
    rng = np.random.default_rng(M)
    locs = np.concatenate([rng.random((3000, 2)), 0.3 + 0.05 * rng.random((400, 2))])   # a dense patch
    J = plan.choose_J_levels(locs, M, max_leaf=40, last_max=last_max)
    assert len(J) == M and J[-1] <= last_max and all(j in (2, 4, 8, 16) for j in J)
    t = O.build_tree(locs, M=M, J=J, r=4)
    assert max(len(o) for o in t.obs) <= 40
    L = int(round(np.log2(np.prod(J))))
    assert plan.cell_occupancy(locs, L - 1).max() > 40


def test_choose_J_levels_errors():
    with pytest.raises(ValueError):
        plan.choose_J_levels(_grid_points(64), 2, max_leaf=1)        # 12 halvings in 2 levels
    with pytest.raises(ValueError):
        plan.choose_J_levels(np.zeros((10, 2)), 3, max_leaf=1)       # coincident points

"""Choice of the number of levels M for a dataset (Sec. 2.5).

The paper recommends M and J as small and r as large as resources allow,
subject to enough resolution; the GPU leaf kernels accept at most
``MRA_MAX_LEAF`` observations per leaf.  ``choose_levels`` returns the smallest
M whose level-M leaves (the 2^M x 2^M midpoint cells of the bounding box) hold
at most ``max_leaf`` observations each.
"""
from __future__ import annotations

import numpy as np


def leaf_occupancy(locs, M: int, bbox=(0.0, 1.0, 0.0, 1.0)) -> np.ndarray:
    """Observations per level-M cell (half-open cells, the last one closed)."""
    x0, x1, y0, y1 = bbox
    g = 1 << M
    ix = np.clip(np.floor((locs[:, 0] - x0) / (x1 - x0) * g).astype(np.int64), 0, g - 1)
    iy = np.clip(np.floor((locs[:, 1] - y0) / (y1 - y0) * g).astype(np.int64), 0, g - 1)
    return np.bincount(ix + g * iy, minlength=g * g)


def choose_levels(locs, max_leaf: int = 64, bbox=(0.0, 1.0, 0.0, 1.0), max_M: int = 12) -> int:
    for M in range(0, max_M + 1):
        if leaf_occupancy(locs, M, bbox).max() <= max_leaf:
            return M
    raise ValueError(f"no M <= {max_M} keeps every leaf at or below {max_leaf} observations")

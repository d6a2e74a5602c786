"""Choice of the partition for a dataset (Sec. 2.2, 2.5, 4.3).

The paper recommends M and J as small and r as large as resources allow,
subject to enough resolution; the GPU leaf kernels accept at most
``MRA_MAX_LEAF`` observations per leaf.  ``choose_levels`` returns the smallest
M whose level-M leaves (the 2^M x 2^M midpoint cells of the bounding box) hold
at most ``max_leaf`` observations each.  ``choose_J_levels`` picks the finest
grid the same way (the fewest midpoint halvings L, alternating x and y) and
spreads its L halvings over a given number of levels with few children at the
coarse levels and more at the fine ones, as Sec. 4.3's (2, 2, 4, 8, 8, 16) does.
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


def cell_occupancy(locs, L: int, bbox=(0.0, 1.0, 0.0, 1.0)) -> np.ndarray:
    """Observations per cell of the 2^ceil(L/2) x 2^floor(L/2) grid (L midpoint
    halvings alternating x, y; half-open cells, the last one closed)."""
    x0, x1, y0, y1 = bbox
    gx, gy = 1 << ((L + 1) // 2), 1 << (L // 2)
    ix = np.clip(np.floor((locs[:, 0] - x0) / (x1 - x0) * gx).astype(np.int64), 0, gx - 1)
    iy = np.clip(np.floor((locs[:, 1] - y0) / (y1 - y0) * gy).astype(np.int64), 0, gy - 1)
    return np.bincount(ix + gx * iy, minlength=gx * gy)


def choose_J_levels(locs, M: int, max_leaf: int = 64, bbox=(0.0, 1.0, 0.0, 1.0), max_L: int = 24,
                    last_max: int = 4):
    """(J_1, ..., J_M) for ``mra_config.J_level``: the fewest halvings L whose
    finest cells hold at most ``max_leaf`` observations, spread over M levels:
    J_M as large as ``last_max`` allows (4 for the emulated form, up to 16 for
    the FP64 and 3xTF32 forms) while every level keeps a halving, the rest
    evenly over levels 1..M-1 with the remainder at the finer ones, each
    1 <= log2 J_m <= 4."""
    locs = np.asarray(locs, dtype=np.float64)
    last_bits = int(last_max).bit_length() - 1
    L = next((k for k in range(0, max_L + 1) if cell_occupancy(locs, k, bbox).max() <= max_leaf), None)
    if L is None:
        raise ValueError(f"no grid of at most 2^{max_L} cells keeps every cell at or below {max_leaf}")
    L = max(L, M)                                  # at least one halving per level
    if M == 1:
        bits = [L]
    else:
        b_last = max(1, min(last_bits, L - (M - 1)))
        rest = L - b_last
        base, extra = divmod(rest, M - 1)
        bits = [base + (1 if m >= M - 1 - extra else 0) for m in range(M - 1)] + [b_last]
    if bits[-1] > last_bits or any(b < 1 or b > 4 for b in bits):
        raise ValueError(f"{L} halvings do not fit {M} levels of 2 to 16 children (J_M <= {last_max})")
    return tuple(1 << b for b in bits)

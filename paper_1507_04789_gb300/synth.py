"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only: spatial locations, field values and
prediction points.  It contains none of the multi-resolution approximation's
arithmetic (no covariance evaluation, no partition, no knots), so that the CUDA
path and the CPU oracle can both be fed from it without sharing method code.

Field values are random-Fourier-feature draws (Rahimi & Recht 2007): for a
Matern-nu correlation with the sqrt(2 nu) h / kappa scaling used in Sec. 4
(Eq. mat15 is nu = 1.5; the exponential is nu = 0.5), the spectral measure is a
bivariate Student-t with 2 nu degrees of freedom scaled by 1/kappa, so
    f(s) = sigma * sqrt(2/D) * sum_j cos(w_j . s + b_j),
    w_j = z_j / (kappa * sqrt(chi2_{2nu} / (2 nu))),  b_j ~ U(0, 2 pi),
has covariance sigma^2 * M_nu(|s1 - s2| / kappa) as D grows.  The paper's own
data (the TPW satellite swaths of Sec. 4.3, the 1-D grid draws of Sec. 4.1) are
not available; these draws stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "uniform_locations",
    "rff_field",
    "noisy_observations",
    "swath_locations",
    "grid_points",
    "Workload",
    "workload",
    "WORKLOADS",
    "swath_batch",
]


def uniform_locations(n: int, seed: int, dim: int = 2) -> np.ndarray:
    """n points uniform on [0,1]^dim, float64, row-major (n, dim)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, dim))


def rff_field(locs: np.ndarray, nu: float, kappa: float, sigma2: float,
              seed: int, features: int = 4096) -> np.ndarray:
    """Random-Fourier-feature approximation of a zero-mean GP draw at ``locs``."""
    rng = np.random.default_rng(seed)
    d = locs.shape[1]
    z = rng.standard_normal((features, d))
    chi = rng.chisquare(2.0 * nu, size=features)
    w = z / (kappa * np.sqrt(chi / (2.0 * nu)))[:, None]
    b = rng.uniform(0.0, 2.0 * math.pi, size=features)
    out = np.empty(locs.shape[0])
    amp = math.sqrt(sigma2) * math.sqrt(2.0 / features)
    chunk = max(256, (1 << 22) // features)
    for i in range(0, locs.shape[0], chunk):
        ph = locs[i:i + chunk] @ w.T + b
        out[i:i + chunk] = amp * np.cos(ph).sum(axis=1)
    return out


def noisy_observations(field: np.ndarray, tau2: float, seed: int) -> np.ndarray:
    """field + iid N(0, tau2) measurement error."""
    rng = np.random.default_rng(seed)
    return field + math.sqrt(tau2) * rng.standard_normal(field.shape[0])


def swath_locations(n: int, n_swaths: int, width: float, seed: int,
                    drop: float = 0.3, angle: float | None = None,
                    segment: float | None = None) -> np.ndarray:
    """Satellite-style swaths with gaps on [0,1]^2.

    ``n_swaths`` parallel strips of the given width at a common angle (random
    if ``angle`` is None) with random offsets; each strip (or, if ``segment`` is
    given, each segment of that length along a strip) is dropped with
    probability ``drop``.  Points are uniform on the union of the kept pieces
    (rejection sampling), so leaf occupancy is very uneven, as in swath data.
    """
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, math.pi) if angle is None else angle
    u = np.array([math.cos(th), math.sin(th)])      # along-swath direction
    v = np.array([-math.sin(th), math.cos(th)])     # across-swath direction
    # offsets of swath centre lines along v, covering the unit square
    proj = np.array([0.0, 1.0, 1.0, 0.0]) * v[0] + np.array([0.0, 0.0, 1.0, 1.0]) * v[1]
    lo, hi = proj.min(), proj.max()
    offs = rng.uniform(lo, hi, size=n_swaths)
    keep_sw = rng.random(n_swaths) >= drop
    if not keep_sw.any():
        keep_sw[0] = True
    seg_keep = None
    if segment is not None:
        n_seg = int(math.ceil(2.0 / segment)) + 1
        seg_keep = rng.random((n_swaths, n_seg)) >= drop
    order = np.argsort(offs)
    so, sk = offs[order], keep_sw[order]
    chunks, have = [], 0
    while have < n:
        cand = rng.random((max(4 * (n - have), 1024), 2))
        cv = cand @ v
        cu = cand @ u
        # nearest swath centre lines below and above each candidate (sorted offsets)
        j = np.searchsorted(so, cv)
        inside = np.zeros(cand.shape[0], dtype=bool)
        for jj in (np.clip(j - 1, 0, len(so) - 1), np.clip(j, 0, len(so) - 1)):
            hit = (np.abs(cv - so[jj]) <= 0.5 * width) & sk[jj]
            if seg_keep is not None:
                si = np.clip(((cu + 1.0) / segment).astype(np.int64), 0, seg_keep.shape[1] - 1)
                hit &= seg_keep[order[jj], si]
            inside |= hit
        acc = cand[inside]
        chunks.append(acc)
        have += acc.shape[0]
    out = np.concatenate(chunks, axis=0)
    return out[:n].copy()


def grid_points(g: int) -> np.ndarray:
    """g x g cell-centred grid on [0,1]^2 (prediction grids)."""
    c = (np.arange(g) + 0.5) / g
    xx, yy = np.meshgrid(c, c, indexing="xy")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


@dataclass(frozen=True)
class Workload:
    """One synthetic problem: sizes, tree shape and covariance parameters."""
    name: str
    n: int
    M: int
    r: int
    family: str          # "exp" or "matern15"
    sigma2: float
    kappa: float
    tau2: float
    n_pred: int
    seed: int = 0
    J: int = 4
    features: int = 4096     # random Fourier features of the field draw
    # "uniform": locations uniform on [0,1]^2, uniform prediction points;
    # "swath200": 200 parallel swaths of width 0.004 at a common angle drawn from
    # 45 +- 5 degrees, cut into 0.05-long segments each dropped with probability
    # 0.3 (the satellite tracks with gaps of Sec. 4.3's data), prediction points
    # on the cell-centred sqrt(n_pred) x sqrt(n_pred) grid
    layout: str = "uniform"
    nonstat: bool = False    # field times sqrt(g(s)), g(s) = 1 + sin(4 pi s_x) / 2

    def generate(self):
        """Return (locs (n,2), y (n,), plocs (n_pred,2)), all float64."""
        nu = 0.5 if self.family == "exp" else 1.5
        if self.layout == "swath200":
            ang = np.random.default_rng(self.seed + 4).uniform(40.0, 50.0) * math.pi / 180.0
            locs = swath_locations(self.n, 200, 0.004, self.seed, drop=0.3, angle=ang, segment=0.05)
            g = int(round(math.sqrt(self.n_pred)))
            plocs = grid_points(g)
        else:
            locs = uniform_locations(self.n, self.seed)
            plocs = uniform_locations(self.n_pred, self.seed + 3)
        field = rff_field(locs, nu, self.kappa, self.sigma2, self.seed + 1, self.features)
        if self.nonstat:
            field *= np.sqrt(1.0 + 0.5 * np.sin(4.0 * math.pi * locs[:, 0]))
        y = noisy_observations(field, self.tau2, self.seed + 2)
        return locs, y, plocs


WORKLOADS = {
    # n=4096 uniform, exponential (sigma2=1, range 0.05), tau2=0.05, M=3, J=4,
    # r=16 (4x4 grid per region), ~64 observations per leaf, 1024 prediction points.
    "n4096_exp_M3_r16": Workload("n4096_exp_M3_r16", 4096, 3, 16, "exp", 1.0, 0.05, 0.05, 1024),
    # n=2^20 uniform, Matern-1.5 (sigma2=1, range 0.1), tau2=0.01, M=7, J=4,
    # r=64 (8x8 grid per region), ~64 observations per leaf.
    "n1M_matern15_M7_r64": Workload("n1M_matern15_M7_r64", 1 << 20, 7, 64, "matern15", 1.0, 0.1, 0.01, 1 << 14,
                                    features=256),
    # n=2^18 with the same leaf shape: profiling size (a few GB on the device).
    "n256k_matern15_M6_r64": Workload("n256k_matern15_M6_r64", 1 << 18, 6, 64, "matern15", 1.0, 0.1, 0.01, 1 << 12,
                                      features=256),
    # n=2^14 with the same leaf shape (gradient parity size).
    "n16k_matern15_M4_r64": Workload("n16k_matern15_M4_r64", 1 << 14, 4, 64, "matern15", 1.0, 0.1, 0.01, 1024),
    # n=2^24 on 200 diagonal swaths with gaps, exponential (Matern-0.5) with the
    # nonstationary variance, range 0.1, tau2=0.02, M=10, r=64, 2^20 grid points.
    "n16M_swath_M10_r64": Workload("n16M_swath_M10_r64", 1 << 24, 10, 64, "exp", 1.0, 0.1, 0.02, 1 << 20,
                                   features=128, layout="swath200", nonstat=True),
    # the same layout at n=2^18, M=7 (about the same observations per active leaf)
    "n256k_swath_M7_r64": Workload("n256k_swath_M7_r64", 1 << 18, 7, 64, "exp", 1.0, 0.1, 0.02, 1 << 12,
                                   features=128, layout="swath200", nonstat=True),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def swath_batch(ndata: int = 64, seed: int = 0, n_min: float = 1e4, n_max: float = 1e6,
                width: float = 0.02, drop: float = 0.3, features: int = 256):
    """Independent swath datasets of log-uniform size (the ragged batch workload).

    Dataset i: n_i = floor(10^U(log10 n_min, log10 n_max)) locations on
    K_i ~ U{8..32} parallel swaths of the given width at a common random angle,
    each swath dropped with probability ``drop``; field = exponential-covariance
    draw with sigma2 = 1 and range kappa_i ~ U(0.02, 0.3), plus N(0, 0.05) noise.
    Returns a list of dicts with locs, y, kappa, sigma2, tau2.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(ndata):
        n = int(10 ** rng.uniform(math.log10(n_min), math.log10(n_max)))
        k = int(rng.integers(8, 33))
        kappa = float(rng.uniform(0.02, 0.3))
        s = int(rng.integers(0, 2 ** 31 - 1))
        locs = swath_locations(n, k, width, s, drop=drop)
        field = rff_field(locs, 0.5, kappa, 1.0, s + 1, features)
        y = noisy_observations(field, 0.05, s + 2)
        out.append({"locs": locs, "y": y, "kappa": kappa, "sigma2": 1.0, "tau2": 0.05})
    return out

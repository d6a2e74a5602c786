"""Independent dense checkers for the M-RA oracle.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; it shares no code with the CUDA library.

* ``exact_*`` : the exact Gaussian process (the 0-RA of Sec. 2.4): dense
  Cholesky of C0(S, S) + tau2 I, Gaussian log-likelihood and simple kriging
  (Sec. 2.1).
* ``bruteforce_cov`` : the M-RA covariance C_M assembled densely from the
  process definition, Eqs. (mra1) and (msadetails) of Sec. 2.3 with reading R2
  (v_{m+1} vanishes between different regions at resolution m+1), and Sec. 2.4
  (C_M(s1, s2) = sum_{l <= m*} b_l(s1)' K_l b_l(s2) when s1, s2 last share a
  region at resolution m* < M, and C0(s1, s2) inside one leaf).  It never runs
  the prior/posterior recursions of Sec. 3, so agreement with them checks those
  recursions.  Dense in all points: meant for n up to a few hundred.

The checkers import nothing from ``mra_oracle``; they read only the knots and
the bounding box of the tree they are given: their covariance ``c0`` is the general Matern
correlation through the modified Bessel function K_nu (scipy.special.kv),
which reduces to the exponential at nu = 1/2 and to Eq. (mat15) at nu = 3/2,
and their point locator ``cell_index`` works on the integer cell grid of each
level (the cell coordinates' bits regrouped into per-level child digits), not
by descending the partition.  For level-varying J (reading R18) the level-m
grid is 2^ceil(L/2) x 2^floor(L/2) cells, L = log2(J_1 ... J_m): the halvings
alternate x, y, x, ... over the whole sequence.  A mistake in the oracle's own C0 or partition therefore shows up
as a disagreement with these checkers.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial.distance import cdist
from scipy.special import gamma, kv

__all__ = ["exact_loglik", "exact_predict", "bruteforce_cov", "bruteforce_loglik",
           "bruteforce_predict", "bruteforce_predict_joint", "gaussian_loglik", "kriging", "c0", "matern",
           "cell_index"]

NU = {"exp": 0.5, "matern15": 1.5}


def matern(h, nu):
    """Matern correlation 2^(1-nu)/Gamma(nu) (sqrt(2 nu) h)^nu K_nu(sqrt(2 nu) h),
    h = distance / range (the parameterisation of Eq. mat15 at nu = 3/2); 1 at h = 0."""
    h = np.asarray(h, dtype=np.float64)
    x = math.sqrt(2.0 * nu) * h
    with np.errstate(invalid="ignore", over="ignore"):
        rho = (2.0 ** (1.0 - nu) / gamma(nu)) * x ** nu * kv(nu, x)
    return np.where(x == 0.0, 1.0, rho)


def c0(X1, X2, theta, family, nonstat=False):
    """C0(X1, X2) = sigma2 rho(|s1 - s2| / range), optionally times the
    nonstationary variance factor sqrt(g(s1) g(s2)), g(s) = 1 + sin(4 pi s_x) / 2;
    theta = (sigma2, range) or, for family "matern", (sigma2, range, nu)."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    nu = theta[2] if family == "matern" else NU[family]
    C = theta[0] * matern(cdist(X1, X2) / theta[1], nu)
    if nonstat:
        s1 = np.sqrt(1.0 + 0.5 * np.sin(4.0 * math.pi * X1[:, 0]))
        s2 = np.sqrt(1.0 + 0.5 * np.sin(4.0 * math.pi * X2[:, 0]))
        C = C * s1[:, None] * s2[None, :]
    return C


def _J(J, k):
    return int(J) if np.isscalar(J) else int(J[k - 1])


def cell_index(pts, bbox, J, m, dim):
    """Index of the level-m region holding each point: the integer cell (the
    box cut into J_1 ... J_m equal parts in 1-D; in 2-D into 2^ceil(L/2) x
    2^floor(L/2) cells, L = log2(J_1 ... J_m); the last cell closed at the box
    maximum), the cell coordinates' bits then read as per-level child digits
    j = c_x + s_x c_y (x bits first, coarse levels in the high bits)."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, dim)
    if dim == 1:
        x0, x1 = bbox
        k = 1
        for l in range(1, m + 1):
            k *= _J(J, l)
        return np.clip(np.floor((pts[:, 0] - x0) / (x1 - x0) * k), 0, k - 1).astype(np.int64)
    x0, x1, y0, y1 = bbox
    L = [0]
    for l in range(1, m + 1):
        L.append(L[-1] + int(round(math.log2(_J(J, l)))))
    NX, NY = (L[m] + 1) // 2, L[m] // 2
    ix = np.clip(np.floor((pts[:, 0] - x0) / (x1 - x0) * 2 ** NX), 0, 2 ** NX - 1).astype(np.int64)
    iy = np.clip(np.floor((pts[:, 1] - y0) / (y1 - y0) * 2 ** NY), 0, 2 ** NY - 1).astype(np.int64)
    out = np.zeros(pts.shape[0], dtype=np.int64)
    for l in range(1, m + 1):
        a = (L[l] + 1) // 2 - (L[l - 1] + 1) // 2          # x halvings of level l
        b = L[l] // 2 - L[l - 1] // 2                      # y halvings
        cx = (ix >> (NX - (L[l] + 1) // 2)) & ((1 << a) - 1)
        cy = (iy >> (NY - L[l] // 2)) & ((1 << b) - 1)
        out = out * _J(J, l) + cx + (cy << a)
    return out


def gaussian_loglik(C, y):
    """log N(y; 0, C) with a dense Cholesky factor."""
    n = y.shape[0]
    L = np.linalg.cholesky(C)
    z = np.linalg.solve(L, y)
    return -np.sum(np.log(np.diag(L))) - 0.5 * z @ z - 0.5 * n * math.log(2.0 * math.pi)


def kriging(C_SS, C_PS, c_PP, y):
    """Simple-kriging mean and variance given the data covariance C_SS."""
    W = np.linalg.solve(C_SS, C_PS.T)
    return C_PS @ np.linalg.solve(C_SS, y), c_PP - np.sum(C_PS * W.T, axis=1)


def _ct(theta):
    """C0's parameters from theta = (sigma2, range, tau2[, nu])."""
    return (theta[0], theta[1]) + ((theta[3],) if len(theta) > 3 else ())


def exact_loglik(locs, y, theta, family, nonstat=False):
    C = c0(locs, locs, _ct(theta), family, nonstat) + theta[2] * np.eye(locs.shape[0])
    return gaussian_loglik(C, y)


def exact_predict(locs, y, plocs, theta, family, nonstat=False):
    C = c0(locs, locs, _ct(theta), family, nonstat) + theta[2] * np.eye(locs.shape[0])
    CP = c0(plocs, locs, _ct(theta), family, nonstat)
    cPP = np.diag(c0(plocs, plocs, _ct(theta), family, nonstat))
    return kriging(C, CP, cPP, y)


def bruteforce_cov(tree, pts, theta, family, nonstat=False):
    """C_M(pts, pts) from the definition of the M-RA process (Sec. 2.3)."""
    J, M, dim = tree.J, tree.M, tree.dim
    nreg = [1]
    for l in range(1, M + 1):
        nreg.append(nreg[-1] * _J(J, l))
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, dim)
    npts = pts.shape[0]
    # Z = the requested points followed by every knot of every internal region
    knot_slices = {}
    Z = [pts]
    off = npts
    for m in range(M):
        for i in range(nreg[m]):
            q = tree.knots[m][i]
            knot_slices[(m, i)] = np.arange(off, off + q.shape[0])
            Z.append(q)
            off += q.shape[0]
    Z = np.concatenate(Z, axis=0)
    # region of every point of Z at every level, by location (Sec. 2.2)
    reg = np.zeros((M + 1, Z.shape[0]), dtype=np.int64)
    for m in range(1, M + 1):
        reg[m] = cell_index(Z, tree.boxes[0][0], J, m, dim)
    v = c0(Z, Z, theta, family, nonstat)              # v_0 = C0
    CM = np.zeros((npts, npts), dtype=v.dtype)
    P = np.arange(npts)
    for m in range(M):
        vn = np.zeros_like(v)
        for i in range(nreg[m]):
            idx = np.flatnonzero(reg[m] == i)
            q = knot_slices[(m, i)]
            K = np.linalg.inv(v[np.ix_(q, q)])             # K_R = v_m(Q, Q)^{-1}
            b = v[np.ix_(idx, q)]                          # b_R(s) = v_m(s, Q)
            bKb = b @ K @ b.T
            # tau_m contributes b' K b for pairs in the same level-m region
            pin = idx[idx < npts]
            sel = np.searchsorted(idx, pin)
            CM[np.ix_(pin, pin)] += bKb[np.ix_(sel, sel)]
            vn[np.ix_(idx, idx)] = v[np.ix_(idx, idx)] - bKb   # Eq. (msadetails)
        same = reg[m + 1][:, None] == reg[m + 1][None, :]       # reading R2
        v = np.where(same, vn, 0.0)
    CM += v[np.ix_(P, P)]                                       # delta_M term
    return CM


def bruteforce_loglik(prob, theta):
    tree = prob.tree
    C = bruteforce_cov(tree, prob.locs, _ct(theta), prob.family, prob.nonstat)
    return gaussian_loglik(C + theta[2] * np.eye(prob.locs.shape[0]), prob.y)


def bruteforce_predict(prob, theta, plocs):
    tree = prob.tree
    n = prob.locs.shape[0]
    allp = np.concatenate([prob.locs, np.asarray(plocs).reshape(-1, tree.dim)], axis=0)
    C = bruteforce_cov(tree, allp, _ct(theta), prob.family, prob.nonstat)
    C_SS = C[:n, :n] + theta[2] * np.eye(n)
    return kriging(C_SS, C[n:, :n], np.diag(C[n:, n:]), prob.y)


def bruteforce_predict_joint(prob, theta, plocs):
    """Joint kriging of y at plocs under the dense C_M: mean and full covariance
    C_M(P, P) - C_M(P, S) (C_M(S, S) + tau2 I)^{-1} C_M(S, P)."""
    tree = prob.tree
    n = prob.locs.shape[0]
    allp = np.concatenate([prob.locs, np.asarray(plocs).reshape(-1, tree.dim)], axis=0)
    C = bruteforce_cov(tree, allp, _ct(theta), prob.family, prob.nonstat)
    C_SS = C[:n, :n] + theta[2] * np.eye(n)
    C_PS = C[n:, :n]
    W = np.linalg.solve(C_SS, C_PS.T)
    return C_PS @ np.linalg.solve(C_SS, prob.y), C[n:, n:] - C_PS @ W

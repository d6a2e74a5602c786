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
"""
from __future__ import annotations

import math

import numpy as np

from . import mra_oracle as O

__all__ = ["exact_loglik", "exact_predict", "bruteforce_cov", "bruteforce_loglik",
           "bruteforce_predict", "gaussian_loglik", "kriging"]


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


def exact_loglik(locs, y, theta, family, nonstat=False):
    C = O.cov(locs, locs, theta[:2], family, nonstat) + theta[2] * np.eye(locs.shape[0])
    return gaussian_loglik(C, y)


def exact_predict(locs, y, plocs, theta, family, nonstat=False):
    C = O.cov(locs, locs, theta[:2], family, nonstat) + theta[2] * np.eye(locs.shape[0])
    CP = O.cov(plocs, locs, theta[:2], family, nonstat)
    cPP = np.diag(O.cov(plocs, plocs, theta[:2], family, nonstat))
    return kriging(C, CP, cPP, y)


def bruteforce_cov(tree, pts, theta, family, nonstat=False):
    """C_M(pts, pts) from the definition of the M-RA process (Sec. 2.3)."""
    J, M, dim = tree.J, tree.M, tree.dim
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, dim)
    npts = pts.shape[0]
    # Z = the requested points followed by every knot of every internal region
    knot_slices = {}
    Z = [pts]
    off = npts
    for m in range(M):
        for i in range(J ** m):
            q = tree.knots[m][i]
            knot_slices[(m, i)] = np.arange(off, off + q.shape[0])
            Z.append(q)
            off += q.shape[0]
    Z = np.concatenate(Z, axis=0)
    # region of every point of Z at every level, by location (Sec. 2.2)
    reg = np.zeros((M + 1, Z.shape[0]), dtype=np.int64)
    for m in range(1, M + 1):
        reg[m] = O.locate(Z, tree.boxes, J, m, dim) if m else 0
    v = O.cov(Z, Z, theta, family, nonstat)           # v_0 = C0
    CM = np.zeros((npts, npts), dtype=v.dtype)
    P = np.arange(npts)
    for m in range(M):
        vn = np.zeros_like(v)
        for i in range(J ** m):
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
    C = bruteforce_cov(tree, prob.locs, theta[:2], prob.family, prob.nonstat)
    return gaussian_loglik(C + theta[2] * np.eye(prob.locs.shape[0]), prob.y)


def bruteforce_predict(prob, theta, plocs):
    tree = prob.tree
    n = prob.locs.shape[0]
    allp = np.concatenate([prob.locs, np.asarray(plocs).reshape(-1, tree.dim)], axis=0)
    C = bruteforce_cov(tree, allp, theta[:2], prob.family, prob.nonstat)
    C_SS = C[:n, :n] + theta[2] * np.eye(n)
    return kriging(C_SS, C[n:, :n], np.diag(C[n:, n:]), prob.y)

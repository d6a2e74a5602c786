"""FP64 CPU oracle of the multi-resolution approximation (M-RA), Katzfuss 2017.

TEST INFRASTRUCTURE ONLY.  This package checks the CUDA path; it is not part of
it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code with
the CUDA library (``paper_1507_04789_gb300/csrc``) and imports nothing from it.

The oracle follows the paper's own statement of the method, in its notation,
with plain numpy/scipy steps (matrix products, inverses, solves) and no
blocking, fusion or reformulation:

* Sec. 2.2: recursive partition into J subregions per level and r knots per
  region; the knots of a leaf are its observations.
* Sec. 3.1, Eq. (priorw): W^l_R = C0(Q_R, Q_{R_l}) - sum_{k<l} W^k_R K_{R_k}
  W^k_{R_l}'; K_R^{-1} = W^m_R (m < M), B^l = W^l_leaf, Sigma_leaf = W^M_leaf.
* Sec. 4.3: measurement error adds sigma_eps^2 I (here ``tau2``) to Sigma_leaf.
* Sec. 3.2, Eqs. (posterior), (mainquantities), (helpquantities): leaf
  A~, omega~ from their definition; A, omega summed over children; K~ =
  (K^{-1} + A^{m,m})^{-1}; A~ = A - A^{k,m} K~ A^{m,l}; omega~ likewise.
* Sec. 3.3: d and u recursions; -2 log L = d + u at the root.
* Sec. 3.4, Prop. 2 and Eq. (bfrecursion): prior prediction quantities U^l,
  L^M, V^P; posterior basis matrices B~^{l,k}; marginal predictive mean and
  variance of y (not of the noisy z, Sec. 4.3); the joint posterior predictive
  covariance that Prop. 2 implies, and draws from it (conditional simulation).

Readings where the paper is silent or garbled:

* R1: the paper's -2 log L omits the Gaussian constant; ``loglik`` returns
  -(d + u)/2 - (n/2) log(2 pi).
* R2: v_{m+1} vanishes between points in different regions at resolution m+1
  (the remainder is made block-independent at the next resolution).
* R4: the sum in V^P runs over k = 0..M-1.
* R5: the prediction mean uses the region's own omega^m_R (Prop. 2).
* R6: the nugget enters only Sigma_leaf (measurement-error form), never a
  knot covariance; predictions are of y.
* R8: knots form a cell-centred g_x x g_y grid inside each region.
* R9: regions split at their midpoint, half-open [lo, mid), [mid, hi]; child
  index j = b_x + 2 b_y in 2-D; in 1-D child j covers the j-th of J equal parts.
* R18: J may vary with the level (Sec. 2.2; Sec. 4.3 takes (J_1, ..., J_6) =
  (2, 2, 4, 8, 8, 16)).  In 2-D every J_m is a power of two and every level-(m-1)
  region splits the same way, into an s_x x s_y grid of equal children (s_x s_y
  = J_m), each side cut by repeated midpoint halving with R9's half-open rule.
  The log2 J_m halvings of level m go one at a time to the axis that has been
  halved fewer times over levels 1..m so far, x on ties (so J = 4 is R9's
  quadtree and (2, 2, 4, 8, 8, 16) ends on a 128 x 128 grid of square leaves);
  child j = c_x + s_x c_y for the child in column c_x and row c_y.
* R10: an empty leaf contributes A~ = 0, omega~ = 0, d = u = 0.
* R17: a draw of eta~_R ~ N(K~_R omega^m_R, K~_R) (Prop. 2) takes the square
  root F_R = L_R^{-T} Lt_R^{-T} of K~_R, with L_R L_R' = K_R^{-1} and
  Lt_R Lt_R' = I + L_R^{-1} A^{m,m}_R L_R^{-T} (both lower Cholesky factors), so
  that F_R F_R' = (K_R^{-1} + A^{m,m}_R)^{-1}; a draw of delta~ in leaf F takes
  the lower Cholesky factor of V^P - L^M Sigma^{-1} L^M' over the leaf's
  prediction points in ascending order of their index.  The standard normals
  are inputs: xi (r per region of levels 0..M-1, complete tree, regions in
  level then index order) and zeta (one per prediction point).
* R12: exponential C0 = s2 exp(-h/kappa); Matern-1.5 C0 = s2 (1 + sqrt3 h/kappa)
  exp(-sqrt3 h/kappa) (Eq. mat15); optional nonstationary variance
  s2 sqrt(g(s1) g(s2)), g(s) = 1 + 0.5 sin(4 pi s_x).
* R13: the Matern family of free smoothness nu (Sec. 4.1's family) in the same
  scaling, s2 2^(1-nu)/Gamma(nu) z^nu K_nu(z), z = sqrt(2 nu) h/kappa, with nu a
  fourth parameter; it equals the exponential at nu = 1/2 and Eq. mat15 at 3/2.

Every routine is written so that the parameters may be complex: the gradient is
the complex-step derivative (Squire & Trapp 1998) of ``loglik``, exact to
rounding.  For that reason the Cholesky factor below is the plain (unconjugated)
L L^T recursion and log-determinants are 2 sum log diag L.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
from scipy.special import gamma as _gamma
from scipy.special import kv as _kv

__all__ = [
    "NotPositiveDefinite",
    "Tree",
    "build_tree",
    "grid_knots",
    "cov",
    "chol",
    "logdet",
    "prior",
    "posterior",
    "loglik",
    "loglik_grad",
    "predict",
    "predict_joint",
    "simulate",
    "xi_offsets",
    "region_terms",
    "posterior_coarse",
]

SQRT3 = math.sqrt(3.0)


class NotPositiveDefinite(ArithmeticError):
    """A matrix the method requires to be positive definite is not."""


# ---------------------------------------------------------------------------
# Sec. 2.2: partition and knots
# ---------------------------------------------------------------------------

@dataclass
class Tree:
    """Recursive partition of the domain (Sec. 2.2) and its knots.

    ``J`` is one number (every level) or the sequence (J_1, ..., J_M) (reading
    R18).  Region i at level m has children J_{m+1} i + j, j = 0..J_{m+1}-1;
    level 0 is the whole bounding box.  ``boxes[m][i]`` is (x0, x1) in 1-D and
    (x0, x1, y0, y1) in 2-D.  ``knots[m][i]`` is the (r_i, d) array of knots for
    m < M; leaves use their observations (``obs[i]`` indexes into the data).
    """
    dim: int
    J: object
    M: int
    boxes: list
    knots: list
    leaf_of: np.ndarray          # leaf index of every observation
    obs: list                    # observation indices per leaf, original order

    def nreg(self, m):
        """Regions at level m: J_1 ... J_m."""
        return n_regions(self.J, m)


def J_at(J, m):
    """J_m: the children of every level-(m-1) region (m >= 1)."""
    return int(J) if np.isscalar(J) else int(J[m - 1])


def n_regions(J, m):
    out = 1
    for k in range(1, m + 1):
        out *= J_at(J, k)
    return out


def halvings(J, m):
    """(a, b): the x and y midpoint halvings of level m in 2-D (reading R18)."""
    nx = ny = 0
    for k in range(1, m + 1):
        jk = J_at(J, k)
        bits = jk.bit_length() - 1
        if jk < 2 or (1 << bits) != jk:
            raise ValueError("in 2-D every J_m must be a power of two >= 2")
        a = b = 0
        for _ in range(bits):
            if nx <= ny:
                nx += 1
                a += 1
            else:
                ny += 1
                b += 1
    return a, b


def _halve(lo, hi, t):
    """The 2^t equal parts of [lo, hi] by t rounds of midpoint halving."""
    parts = [(lo, hi)]
    for _ in range(t):
        nxt = []
        for a, b in parts:
            mid = 0.5 * (a + b)
            nxt.extend([(a, mid), (mid, b)])
        parts = nxt
    return parts


def _child_boxes(box, J, m, dim):
    """Children of a level-(m-1) region, in child order (readings R9, R18)."""
    Jm = J_at(J, m)
    if dim == 1:
        x0, x1 = box
        w = x1 - x0
        return [(x0 + j * w / Jm, x0 + (j + 1) * w / Jm) for j in range(Jm)]
    a, b = halvings(J, m)
    x0, x1, y0, y1 = box
    xs, ys = _halve(x0, x1, a), _halve(y0, y1, b)
    return [xs[cx] + ys[cy] for cy in range(len(ys)) for cx in range(len(xs))]


def _child_index(pts, boxes_of_pts, J, m, dim):
    """Child j of each point inside its current level-(m-1) box (R9, R18)."""
    Jm = J_at(J, m)
    if dim == 1:
        x0, x1 = boxes_of_pts[:, 0], boxes_of_pts[:, 1]
        j = np.floor((pts[:, 0] - x0) * Jm / (x1 - x0)).astype(np.int64)
        return np.clip(j, 0, Jm - 1)
    a, b = halvings(J, m)

    def side(v, lo, hi, t):
        lo, hi = lo.copy(), hi.copy()
        c = np.zeros(v.shape[0], dtype=np.int64)
        for _ in range(t):
            mid = 0.5 * (lo + hi)
            up = v >= mid
            lo = np.where(up, mid, lo)
            hi = np.where(up, hi, mid)
            c = 2 * c + up
        return c

    cx = side(pts[:, 0], boxes_of_pts[:, 0], boxes_of_pts[:, 1], a)
    cy = side(pts[:, 1], boxes_of_pts[:, 2], boxes_of_pts[:, 3], b)
    return cx + (1 << a) * cy


def locate(pts, tree_boxes, J, M, dim):
    """Leaf index (level M) of each point, descending the partition."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, dim)
    idx = np.zeros(pts.shape[0], dtype=np.int64)
    for m in range(M):
        b = np.asarray(tree_boxes[m], dtype=np.float64).reshape(n_regions(J, m), -1)[idx]
        idx = J_at(J, m + 1) * idx + _child_index(pts, b, J, m + 1, dim)
    return idx


def grid_knots(box, r, dim):
    """Cell-centred equidistant grid of r knots inside ``box`` (reading R8)."""
    if dim == 1:
        x0, x1 = box
        return (x0 + (np.arange(r) + 0.5) * (x1 - x0) / r).reshape(r, 1)
    gx = next(g for g in range(1, r + 1) if r % g == 0 and g * g >= r)  # 8x4 for r = 32
    gy = r // gx
    x0, x1, y0, y1 = box
    xs = x0 + (np.arange(gx) + 0.5) * (x1 - x0) / gx
    ys = y0 + (np.arange(gy) + 0.5) * (y1 - y0) / gy
    xx, yy = np.meshgrid(xs, ys, indexing="xy")   # x fastest
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def build_tree(locs, M, J=4, r=16, bbox=None, knots_fn=None):
    """Partition (Sec. 2.2) with ``r`` grid knots per region, or ``knots_fn``.

    ``J``: children per region, one number or (J_1, ..., J_M) (reading R18).
    ``knots_fn(m, i, box)`` may return any (r_i, d) array of knots for region
    (m, i); it is used for the exactness pins (boundary knots, knots equal to
    the data).
    """
    locs = np.asarray(locs, dtype=np.float64)
    dim = locs.shape[1]
    if not np.isscalar(J):
        J = tuple(int(j) for j in J)
        if len(J) != M:
            raise ValueError("J needs one entry per level 1..M")
    if bbox is None:
        bbox = (0.0, 1.0) if dim == 1 else (0.0, 1.0, 0.0, 1.0)
    boxes = [[tuple(bbox)]]
    for m in range(M):
        nxt = []
        for b in boxes[m]:
            nxt.extend(_child_boxes(b, J, m + 1, dim))
        boxes.append(nxt)
    knots = []
    for m in range(M):
        km = []
        for i, b in enumerate(boxes[m]):
            km.append(np.asarray(knots_fn(m, i, b), dtype=np.float64).reshape(-1, dim)
                      if knots_fn is not None else grid_knots(b, r, dim))
        knots.append(km)
    leaf_of = locate(locs, boxes, J, M, dim)
    nl = n_regions(J, M)
    order = np.argsort(leaf_of, kind="stable")         # original order within a leaf
    cuts = np.searchsorted(leaf_of[order], np.arange(nl + 1))
    obs = [order[cuts[i]:cuts[i + 1]] for i in range(nl)]
    return Tree(dim, J, M, boxes, knots, leaf_of, obs)


def ancestors(m, i, J):
    """(level, index) of the ancestors R_0, ..., R_m of region (m, i)."""
    out = [(m, i)]
    for l in range(m, 0, -1):
        i //= J_at(J, l)
        out.append((l - 1, i))
    return out[::-1]


# ---------------------------------------------------------------------------
# Covariance function C0 (Sec. 2.1; Eq. mat15; Sec. 4.2, 4.3)
# ---------------------------------------------------------------------------

def _dist(X1, X2):
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    diff = X1[:, None, :] - X2[None, :, :]
    return np.sqrt(np.sum(diff * diff, axis=2))


def cov(X1, X2, theta, family, nonstat=False):
    """C0(X1, X2) for theta = (sigma2, kappa) or, for the family "matern" of
    free smoothness, (sigma2, kappa, nu); complex sigma2, kappa allowed."""
    sigma2, kappa = theta[0], theta[1]
    h = _dist(X1, X2) / kappa
    if family == "exp":
        rho = np.exp(-h)
    elif family == "matern15":
        rho = (1.0 + SQRT3 * h) * np.exp(-SQRT3 * h)
    elif family == "matern":
        # Sec. 4.1's Matern family in Eq. mat15's scaling: 2^(1-nu)/Gamma(nu) z^nu K_nu(z),
        # z = sqrt(2 nu) h; K_nu from the library (complex z for the complex step)
        nu = float(np.real(theta[2]))
        z = math.sqrt(2.0 * nu) * h
        zs = np.where(z == 0.0, 1.0, z)
        rho = np.where(z == 0.0, 1.0, (2.0 ** (1.0 - nu) / _gamma(nu)) * zs ** nu * _kv(nu, zs))
    else:
        raise ValueError(f"unknown covariance family {family!r}")
    C = sigma2 * rho
    if nonstat:
        g1 = 1.0 + 0.5 * np.sin(4.0 * math.pi * np.asarray(X1)[:, 0])
        g2 = 1.0 + 0.5 * np.sin(4.0 * math.pi * np.asarray(X2)[:, 0])
        C = C * np.sqrt(np.outer(g1, g2))
    return C


# ---------------------------------------------------------------------------
# Plain dense helpers
# ---------------------------------------------------------------------------

def chol(A):
    """Lower factor L with L L^T = A by the column recursion (no conjugation)."""
    A = np.asarray(A)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        s = A[j, j] - L[j, :j] @ L[j, :j]
        if np.real(s) <= 0.0 or not np.isfinite(s):
            raise NotPositiveDefinite(f"pivot {j} of {n} is {s}")
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def logdet(A):
    """log|A| = 2 sum log diag chol(A)."""
    if A.shape[0] == 0:
        return 0.0
    return 2.0 * np.sum(np.log(np.diag(chol(A))))


def inv(A):
    return np.linalg.inv(A)


def solve(A, B):
    return np.linalg.solve(A, B)


# ---------------------------------------------------------------------------
# Sec. 3.1: prior quantities
# ---------------------------------------------------------------------------

@dataclass
class Prior:
    W: dict = field(default_factory=dict)     # (m, i) -> [W^0_R, ..., W^m_R]
    K: dict = field(default_factory=dict)     # (m, i) -> K_R (m < M)
    Sigma: dict = field(default_factory=dict)  # leaf i -> Sigma_leaf (+ tau2 I)


def _region_points(tree, locs, m, i):
    return tree.knots[m][i] if m < tree.M else locs[tree.obs[i]]


def _in_scope(tree, m, i, subtree):
    """True if region (m, i) belongs to ``subtree`` = (k, idx) or its ancestors."""
    if subtree is None:
        return True
    k, idx = subtree
    if m <= k:
        return i == ancestors(k, idx, tree.J)[m][1]
    return ancestors(m, i, tree.J)[k][1] == idx


def prior(tree, locs, theta, family, tau2, nonstat=False, subtree=None, levels=None):
    """Eq. (priorw) for every region, top-down; Sec. 4.3 nugget on Sigma_leaf.
    ``levels``: only the levels 0..levels."""
    J, M = tree.J, tree.M
    P = Prior()
    for m in range(M + 1 if levels is None else levels + 1):
        for i in range(tree.nreg(m)):
            if not _in_scope(tree, m, i, subtree):
                continue
            anc = ancestors(m, i, J)
            Q = _region_points(tree, locs, m, i)
            Wl = []
            for l, (ml, il) in enumerate(anc):
                Ql = Q if l == m else tree.knots[ml][il]
                X = cov(Q, Ql, theta, family, nonstat)
                for k in range(l):
                    Wk_Rl = Wl[k] if l == m else P.W[(ml, il)][k]
                    X = X - Wl[k] @ P.K[anc[k]] @ Wk_Rl.T
                Wl.append(X)
            P.W[(m, i)] = Wl
            if m < M:
                P.K[(m, i)] = inv(Wl[m])
            else:
                P.Sigma[i] = Wl[M] + tau2 * np.eye(Q.shape[0])
    return P


# ---------------------------------------------------------------------------
# Sec. 3.2 / 3.3: posterior quantities and the likelihood
# ---------------------------------------------------------------------------

@dataclass
class Posterior:
    A: dict = field(default_factory=dict)       # (m, i) -> {(k, l): A^{k,l}_R}, k, l <= m
    omega: dict = field(default_factory=dict)   # (m, i) -> [omega^0_R, ..., omega^m_R]
    Kt: dict = field(default_factory=dict)      # (m, i) -> K~_R
    d: dict = field(default_factory=dict)       # (m, i) -> d_R
    u: dict = field(default_factory=dict)       # (m, i) -> u_R


def _dims(tree, m, i):
    """Knot counts r_{R_0}, ..., r_{R_{m}} along the ancestor chain (internal)."""
    return [tree.knots[l][il].shape[0] for l, il in ancestors(m, i, tree.J)]


def posterior(tree, locs, y, P, subtree=None):
    """Leaves from the definition, then Eqs. (mainquantities)-(helpquantities)."""
    J, M = tree.J, tree.M
    Q = Posterior()
    At, wt = {}, {}          # A~ and omega~ handed to the parent
    dtype = np.result_type(*[P.Sigma[i] for i in P.Sigma]) if P.Sigma else np.float64
    for i in range(tree.nreg(M)):
        if not _in_scope(tree, M, i, subtree):
            continue
        B = P.W[(M, i)][:M]
        yi = y[tree.obs[i]]
        S = P.Sigma[i]
        if S.shape[0] == 0:                       # R10: empty leaf
            rs = _dims(tree, M - 1, i // J_at(J, M)) if M > 0 else []
            At[(M, i)] = {(k, l): np.zeros((rs[k], rs[l]), dtype=dtype)
                          for k in range(M) for l in range(M)}
            wt[(M, i)] = [np.zeros(rs[k], dtype=dtype) for k in range(M)]
            Q.d[(M, i)] = 0.0
            Q.u[(M, i)] = 0.0
            continue
        SiB = [solve(S, Bl) for Bl in B]
        Siy = solve(S, yi)
        At[(M, i)] = {(k, l): B[k].T @ SiB[l] for k in range(M) for l in range(M)}
        wt[(M, i)] = [B[k].T @ Siy for k in range(M)]
        Q.d[(M, i)] = logdet(S)
        Q.u[(M, i)] = yi @ Siy
    for m in range(M - 1, -1, -1):
        Jc = J_at(J, m + 1)
        for i in range(tree.nreg(m)):
            if not _in_scope(tree, m, i, subtree):
                continue
            kids = [(m + 1, Jc * i + j) for j in range(Jc) if (m + 1, Jc * i + j) in At]
            A = {(k, l): sum(At[c][(k, l)] for c in kids) for k in range(m + 1) for l in range(m + 1)}
            om = [sum(wt[c][k] for c in kids) for k in range(m + 1)]
            _post_region(P, Q, At, wt, m, i, A, om, sum(Q.d[c] for c in kids), sum(Q.u[c] for c in kids))
    return Q


def _post_region(P, Q, At, wt, m, i, A, om, dkids, ukids):
    """One region of Eqs. (posterior), (helpquantities) and the d, u recursion
    of Sec. 3.3, given its A^{k,l}, omega^k (Eq. mainquantities) and the sums
    of its children's d and u."""
    Kinv = P.W[(m, i)][m]
    Kt = inv(Kinv + A[(m, m)])
    Q.A[(m, i)] = A
    Q.omega[(m, i)] = om
    Q.Kt[(m, i)] = Kt
    At[(m, i)] = {(k, l): A[(k, l)] - A[(k, m)] @ Kt @ A[(m, l)]
                  for k in range(m) for l in range(m)}
    wt[(m, i)] = [om[k] - A[(k, m)] @ Kt @ om[m] for k in range(m)]
    Q.d[(m, i)] = logdet(Kinv + A[(m, m)]) - logdet(Kinv) + dkids
    Q.u[(m, i)] = -om[m] @ Kt @ om[m] + ukids


def posterior_coarse(tree, P, s, A_s, omega_s, dkids_s, ukids_s):
    """The posterior of levels s..0 (Eqs. mainquantities, posterior,
    helpquantities; Sec. 3.3) from every level-s region's A^{k,l}, omega^k
    (k, l <= s) and its children's d, u sums, as the level-s subtrees of a
    sharded evaluation hand them up (Sec. 3.5).  P needs levels 0..s."""
    J = tree.J
    Q = Posterior()
    At, wt = {}, {}
    for i in range(tree.nreg(s)):
        _post_region(P, Q, At, wt, s, i, A_s[i], omega_s[i], dkids_s[i], ukids_s[i])
    for m in range(s - 1, -1, -1):
        Jc = J_at(J, m + 1)
        for i in range(tree.nreg(m)):
            kids = [(m + 1, Jc * i + j) for j in range(Jc)]
            A = {(k, l): sum(At[c][(k, l)] for c in kids) for k in range(m + 1) for l in range(m + 1)}
            om = [sum(wt[c][k] for c in kids) for k in range(m + 1)]
            _post_region(P, Q, At, wt, m, i, A, om, sum(Q.d[c] for c in kids), sum(Q.u[c] for c in kids))
    return Q


@dataclass
class Problem:
    """Inputs of one M-RA evaluation."""
    locs: np.ndarray
    y: np.ndarray
    M: int
    J: object = 4                 # one number, or (J_1, ..., J_M) (reading R18)
    r: int = 16
    family: str = "exp"
    nonstat: bool = False
    bbox: tuple | None = None
    knots_fn: object = None
    _tree: Tree | None = None

    @property
    def tree(self) -> Tree:
        if self._tree is None:
            self._tree = build_tree(self.locs, self.M, self.J, self.r, self.bbox, self.knots_fn)
        return self._tree


def _split_theta(theta):
    """theta = (sigma2, kappa, tau2) or (sigma2, kappa, tau2, nu): C0's parameters and tau2."""
    sigma2, kappa, tau2 = theta[0], theta[1], theta[2]
    if len(theta) > 3:
        return (sigma2, kappa, theta[3]), tau2
    return (sigma2, kappa), tau2


def loglik(prob: Problem, theta, subtree=None, return_state=False):
    """Sec. 3.3: loglik = -(d + u)/2 - (n/2) log(2 pi)  (reading R1)."""
    tree = prob.tree
    th, tau2 = _split_theta(theta)
    P = prior(tree, prob.locs, th, prob.family, tau2, prob.nonstat, subtree)
    Q = posterior(tree, prob.locs, prob.y, P, subtree)
    root = (0, 0)
    n = prob.locs.shape[0]
    ll = -0.5 * (Q.d[root] + Q.u[root]) - 0.5 * n * math.log(2.0 * math.pi)
    if return_state:
        return ll, P, Q
    return ll


def region_terms(prob: Problem, theta, m, i):
    """(d_R, u_R) of region (m, i) computed from its own subtree (Sec. 3.3)."""
    tree = prob.tree
    th, tau2 = _split_theta(theta)
    P = prior(tree, prob.locs, th, prob.family, tau2, prob.nonstat, subtree=(m, i))
    Q = posterior(tree, prob.locs, prob.y, P, subtree=(m, i))
    return Q.d[(m, i)], Q.u[(m, i)]


def loglik_grad(prob: Problem, theta, step=1e-30):
    """(loglik, d loglik / d(sigma2, kappa, tau2)) by the complex step; with a
    fourth parameter nu (family "matern") also d/dnu, by central differences
    extrapolated once (Richardson): the library Bessel function takes no
    complex order, and the extrapolated difference is accurate to about 1e-9
    relative."""
    theta = np.asarray(theta, dtype=np.float64)
    ll = loglik(prob, theta)
    g = np.zeros(len(theta))
    for a in range(3):
        tc = theta.astype(np.complex128)
        h = step * max(abs(theta[a]), 1.0)
        tc[a] += 1j * h
        g[a] = np.imag(loglik(prob, tc)) / h
    if len(theta) > 3:
        def cd(e):
            tp, tm = theta.copy(), theta.copy()
            tp[3] += e
            tm[3] -= e
            return (loglik(prob, tp) - loglik(prob, tm)) / (2.0 * e)
        e = 2e-3 * theta[3]
        g[3] = (4.0 * cd(0.5 * e) - cd(e)) / 3.0
    return ll, g


# ---------------------------------------------------------------------------
# Sec. 3.4: spatial prediction (Prop. 2, Eq. bfrecursion)
# ---------------------------------------------------------------------------

def predict(prob: Problem, theta, plocs, state=None):
    """Marginal posterior predictive mean and variance of y at ``plocs``."""
    tree = prob.tree
    J, M = tree.J, tree.M
    th, tau2 = _split_theta(theta)
    if state is None:
        _, P, Q = loglik(prob, theta, return_state=True)
    else:
        P, Q = state
    plocs = np.asarray(plocs, dtype=np.float64).reshape(-1, tree.dim)
    pleaf = locate(plocs, tree.boxes, J, M, tree.dim)
    mean = np.zeros(plocs.shape[0])
    var = np.zeros(plocs.shape[0])
    for f in np.unique(pleaf):
        pidx = np.flatnonzero(pleaf == f)
        SP = plocs[pidx]
        anc = ancestors(M, f, J)
        SF = prob.locs[tree.obs[f]]
        yF = prob.y[tree.obs[f]]
        # prior prediction quantities U^l = v_l(S^P, Q_l), l = 0..M
        U = []
        for l, (ml, il) in enumerate(anc):
            Ql = SF if l == M else tree.knots[ml][il]
            X = cov(SP, Ql, th, prob.family, prob.nonstat)
            for k in range(l):
                X = X - U[k] @ P.K[anc[k]] @ P.W[(ml, il)][k].T
            U.append(X)
        LM = U[M]
        VP = cov(SP, SP, th, prob.family, prob.nonstat)
        for k in range(M):
            VP = VP - U[k] @ P.K[anc[k]] @ U[k].T            # reading R4
        S = P.Sigma[f]
        if S.shape[0]:
            SiL = solve(S, LM.T)                               # Sigma^{-1} L^M'
            SiB = [solve(S, P.W[(M, f)][k]) for k in range(M)]
            mu = LM @ solve(S, yF)
            Psi = np.diag(VP) - np.sum(LM * SiL.T, axis=1)
            Bt = {(M, k): U[k] - LM @ SiB[k] for k in range(M)}   # definition, l = M
        else:
            mu = np.zeros(len(pidx))
            Psi = np.diag(VP).copy()
            Bt = {(M, k): U[k] for k in range(M)}
        for l in range(M - 1, 0, -1):                          # recursion, l = M-1..1
            Rl = anc[l]
            for k in range(l):
                Bt[(l, k)] = Bt[(l + 1, k)] - Bt[(l + 1, l)] @ Q.Kt[Rl] @ Q.A[Rl][(l, k)]
        for m in range(M):
            Rm = anc[m]
            Btm = Bt[(m + 1, m)]
            mu = mu + Btm @ (Q.Kt[Rm] @ Q.omega[Rm][m])        # reading R5
            Psi = Psi + np.sum((Btm @ Q.Kt[Rm]) * Btm, axis=1)
        mean[pidx] = np.real(mu)
        var[pidx] = np.real(Psi)
    return mean, var


# ---------------------------------------------------------------------------
# Sec. 3.4: joint posterior predictive distribution and conditional simulation
# ---------------------------------------------------------------------------

def _joint_leaf(prob, P, Q, th, f, SP):
    """Per leaf f: the terms of Prop. 2 for its prediction points SP.

    Returns (Btm, D, dmean): Btm[m] = B~^{m+1,m} (n_P x r_m) for m < M, the
    covariance D = V^P - L^M Sigma^{-1} L^M' of delta~ (full n_P x n_P) and
    its mean L^M Sigma^{-1} y_F."""
    tree = prob.tree
    J, M = tree.J, tree.M
    anc = ancestors(M, f, J)
    SF = prob.locs[tree.obs[f]]
    yF = prob.y[tree.obs[f]]
    U = []
    for l, (ml, il) in enumerate(anc):
        Ql = SF if l == M else tree.knots[ml][il]
        X = cov(SP, Ql, th, prob.family, prob.nonstat)
        for k in range(l):
            X = X - U[k] @ P.K[anc[k]] @ P.W[(ml, il)][k].T
        U.append(X)
    LM = U[M]
    VP = cov(SP, SP, th, prob.family, prob.nonstat)
    for k in range(M):
        VP = VP - U[k] @ P.K[anc[k]] @ U[k].T                     # reading R4
    S = P.Sigma[f]
    if S.shape[0]:
        D = VP - LM @ solve(S, LM.T)
        dmean = LM @ solve(S, yF)
        Bt = {(M, k): U[k] - LM @ solve(S, P.W[(M, f)][k]) for k in range(M)}
    else:
        D = VP
        dmean = np.zeros(SP.shape[0])
        Bt = {(M, k): U[k] for k in range(M)}
    for l in range(M - 1, 0, -1):
        Rl = anc[l]
        for k in range(l):
            Bt[(l, k)] = Bt[(l + 1, k)] - Bt[(l + 1, l)] @ Q.Kt[Rl] @ Q.A[Rl][(l, k)]
    return [Bt[(m + 1, m)] for m in range(M)], D, dmean


def predict_joint(prob: Problem, theta, plocs, state=None):
    """Joint posterior predictive distribution of y at ``plocs`` (Prop. 2).

    Prop. 2 writes y(S^P_F) | data = sum_{m<M} B~^{m+1,m}_F eta~_{R_m} + delta~_F
    with independent eta~_R ~ N(K~_R omega^m_R, K~_R) shared by every leaf under
    R and independent delta~_F per leaf, so for s1 in leaf F1 and s2 in F2
        Cov(s1, s2) = sum_{m<M: R_m(F1) = R_m(F2)} B~^{m+1,m}(s1) K~_{R_m} B~^{m+1,m}(s2)'
                      + 1[F1 = F2] D_F(s1, s2).
    Returns (mean, cov) with cov the full np x np matrix."""
    tree = prob.tree
    J, M = tree.J, tree.M
    th, tau2 = _split_theta(theta)
    if state is None:
        _, P, Q = loglik(prob, theta, return_state=True)
    else:
        P, Q = state
    plocs = np.asarray(plocs, dtype=np.float64).reshape(-1, tree.dim)
    npts = plocs.shape[0]
    pleaf = locate(plocs, tree.boxes, J, M, tree.dim)
    mean = np.zeros(npts)
    cov_out = np.zeros((npts, npts))
    terms = {}
    for f in np.unique(pleaf):
        pidx = np.flatnonzero(pleaf == f)
        Btm, D, dmean = _joint_leaf(prob, P, Q, th, f, plocs[pidx])
        anc = ancestors(M, f, J)
        mu = dmean.copy()
        for m in range(M):
            Rm = anc[m]
            mu = mu + Btm[m] @ (Q.Kt[Rm] @ Q.omega[Rm][m])           # reading R5
        mean[pidx] = np.real(mu)
        cov_out[np.ix_(pidx, pidx)] += np.real(D)
        terms[f] = (pidx, Btm, anc)
    leaves = list(terms)
    for f1 in leaves:
        p1, B1, a1 = terms[f1]
        for f2 in leaves:
            p2, B2, a2 = terms[f2]
            for m in range(M):
                if a1[m] != a2[m]:
                    break                          # no common ancestor below level m
                cov_out[np.ix_(p1, p2)] += np.real(B1[m] @ Q.Kt[a1[m]] @ B2[m].T)
    return mean, cov_out


def xi_offsets(tree):
    """Start of region (m, i)'s r_i normals in a draw's xi vector (reading R17):
    regions of levels 0..M-1 in level, then index order."""
    off, pos = {}, 0
    for m in range(tree.M):
        for i in range(tree.nreg(m)):
            off[(m, i)] = pos
            pos += tree.knots[m][i].shape[0]
    return off, pos


def simulate(prob: Problem, theta, plocs, xi, zeta, state=None):
    """Draws from the joint posterior predictive distribution (Prop. 2) given the
    standard normals xi (nsim x len) and zeta (nsim x np), reading R17:
        eta~_R = K~_R omega^m_R + F_R xi_R,  F_R = L_R^{-T} Lt_R^{-T},
        delta~_F = L^M Sigma^{-1} y_F + chol(D_F) zeta_F,
        y*(S^P_F) = sum_{m<M} B~^{m+1,m}_F eta~_{R_m} + delta~_F."""
    tree = prob.tree
    J, M = tree.J, tree.M
    th, tau2 = _split_theta(theta)
    if state is None:
        _, P, Q = loglik(prob, theta, return_state=True)
    else:
        P, Q = state
    plocs = np.asarray(plocs, dtype=np.float64).reshape(-1, tree.dim)
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    zeta = np.atleast_2d(np.asarray(zeta, dtype=np.float64))
    nsim = xi.shape[0]
    off, _ = xi_offsets(tree)
    # the square roots F_R of K~_R, and the means K~_R omega^m_R
    F, mK = {}, {}
    for (m, i), Kt in Q.Kt.items():
        L = chol(P.W[(m, i)][m])                      # L L' = K^{-1}
        Li = np.linalg.inv(L)
        Lt = chol(np.eye(L.shape[0]) + Li @ Q.A[(m, i)][(m, m)] @ Li.T)
        F[(m, i)] = Li.T @ np.linalg.inv(Lt).T
        mK[(m, i)] = Kt @ Q.omega[(m, i)][m]
    pleaf = locate(plocs, tree.boxes, J, M, tree.dim)
    draws = np.zeros((nsim, plocs.shape[0]))
    for f in np.unique(pleaf):
        pidx = np.flatnonzero(pleaf == f)
        Btm, D, dmean = _joint_leaf(prob, P, Q, th, f, plocs[pidx])
        Lc = chol(D)
        anc = ancestors(M, f, J)
        for s in range(nsim):
            v = dmean + Lc @ zeta[s, pidx]
            for m in range(M):
                R = anc[m]
                xr = xi[s, off[R]:off[R] + F[R].shape[1]]
                v = v + Btm[m] @ (mK[R] + F[R] @ xr)
            draws[s, pidx] = np.real(v)
    return draws

"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test ties the oracle to something other than itself: the exact Gaussian
process, a dense construction of the M-RA covariance straight from the process
definition, closed forms and invariances.  None needs a GPU.
"""
import math

import numpy as np
import pytest

from oracle import exact as E
from oracle import mra_oracle as O

TH_EXP = (1.0, 0.2, 0.1)
TH_M15 = (1.3, 0.15, 0.05)


def _data(n, seed, dim=2):
    rng = np.random.default_rng(seed)
    return rng.random((n, dim)), rng.standard_normal(n)


# ---- P1: M = 0 is the exact GP (Sec. 2.4) --------------------------------------

@pytest.mark.parametrize("family,theta", [("exp", TH_EXP), ("matern15", TH_M15)])
def test_p1_zero_levels_is_exact_gp(family, theta):
    locs, y = _data(80, 1)
    plocs, _ = _data(15, 2)
    p = O.Problem(locs, y, M=0, r=4, family=family)
    assert O.loglik(p, theta) == pytest.approx(E.exact_loglik(locs, y, theta, family), rel=1e-12)
    mu, var = O.predict(p, theta, plocs)
    mu0, var0 = E.exact_predict(locs, y, plocs, theta, family)
    np.testing.assert_allclose(mu, mu0, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(var, var0, rtol=1e-10, atol=1e-12)


# ---- P2: knots equal to the data at resolution 0 make the M-RA exact (Sec. 2.4) --

def test_p2_data_knots_reproduce_exact_gp():
    locs, y = _data(40, 3)
    plocs, _ = _data(12, 4)
    theta = (1.0, 0.3, 0.2)

    def knots(m, i, box):
        return locs if m == 0 else O.grid_knots(box, 4, 2)

    p = O.Problem(locs, y, M=2, J=4, family="exp", knots_fn=knots)
    assert O.loglik(p, theta) == pytest.approx(E.exact_loglik(locs, y, theta, "exp"), rel=1e-9)
    mu, var = O.predict(p, theta, plocs)
    mu0, var0 = E.exact_predict(locs, y, plocs, theta, "exp")
    np.testing.assert_allclose(mu, mu0, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(var, var0, rtol=1e-7, atol=1e-8)


# ---- P3: 1-D exponential with knots on child boundaries is exact (Fig. 1, Sec. 2.5)

@pytest.mark.parametrize("tau2", [0.0, 0.05])
def test_p3_boundary_knots_exact_in_1d(tau2):
    rng = np.random.default_rng(5)
    n, J, M = 54, 3, 3
    locs = rng.random((n, 1))
    y = rng.standard_normal(n)
    plocs = rng.random((20, 1))
    theta = (1.0, 0.1, tau2)

    def knots(m, i, box):
        x0, x1 = box
        return np.array([[x0 + j * (x1 - x0) / J] for j in range(1, J)])

    p = O.Problem(locs, y, M=M, J=J, family="exp", knots_fn=knots)
    assert O.loglik(p, theta) == pytest.approx(E.exact_loglik(locs, y, theta, "exp"), rel=1e-10)
    mu, var = O.predict(p, theta, plocs)
    mu0, var0 = E.exact_predict(locs, y, plocs, theta, "exp")
    np.testing.assert_allclose(mu, mu0, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(var, var0, rtol=1e-8, atol=1e-10)


def test_p3_interior_knots_are_not_exact():
    """Control for P3: the same tree with interior knots is only an approximation."""
    rng = np.random.default_rng(5)
    locs = rng.random((54, 1))
    y = rng.standard_normal(54)
    def knots(m, i, box):
        x0, x1 = box
        return np.array([[x0 + 0.2 * (x1 - x0)], [x0 + 0.7 * (x1 - x0)]])

    p = O.Problem(locs, y, M=3, J=3, family="exp", knots_fn=knots)
    theta = (1.0, 0.1, 0.05)
    assert abs(O.loglik(p, theta) - E.exact_loglik(locs, y, theta, "exp")) > 1e-4


# ---- P4: recursions of Sec. 3 == dense C_M from the definition (Sec. 2.3) ------

@pytest.mark.parametrize("M,r,family,nonstat", [
    (1, 4, "exp", False), (2, 9, "matern15", False), (3, 4, "exp", False),
    (2, 16, "exp", False), (3, 9, "matern15", True),
])
def test_p4_recursions_match_bruteforce(M, r, family, nonstat):
    locs, y = _data(220, 10 + M + r)
    plocs, _ = _data(25, 20 + M)
    theta = TH_M15 if family == "matern15" else TH_EXP
    p = O.Problem(locs, y, M=M, r=r, family=family, nonstat=nonstat)
    assert O.loglik(p, theta) == pytest.approx(E.bruteforce_loglik(p, theta), rel=1e-11)
    mu, var = O.predict(p, theta, plocs)
    mu_b, var_b = E.bruteforce_predict(p, theta, plocs)
    np.testing.assert_allclose(mu, mu_b, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(var, var_b, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("J,r,family", [((2, 8), 4, "exp"), ((2, 2, 4), 9, "matern15"), ((16, 2), 4, "exp"),
                                         ((8,), 9, "matern15")])
def test_p4_level_varying_J_matches_bruteforce(J, r, family):
    """P4 on partitions with level-varying J (reading R18): the recursions of
    Sec. 3 against the dense C_M of the process definition."""
    locs, y = _data(220, 40 + sum(J))
    plocs, _ = _data(25, 41 + sum(J))
    theta = TH_M15 if family == "matern15" else TH_EXP
    p = O.Problem(locs, y, M=len(J), J=J, r=r, family=family)
    assert O.loglik(p, theta) == pytest.approx(E.bruteforce_loglik(p, theta), rel=1e-11)
    mu, var = O.predict(p, theta, plocs)
    mu_b, var_b = E.bruteforce_predict(p, theta, plocs)
    np.testing.assert_allclose(mu, mu_b, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(var, var_b, rtol=1e-8, atol=1e-10)
    mean, cov = O.predict_joint(p, theta, plocs)
    mb, cb = E.bruteforce_predict_joint(p, theta, plocs)
    np.testing.assert_allclose(cov, cb, rtol=1e-8, atol=1e-10)


def test_p2_level_varying_J_data_knots_exact():
    """P2 on a level-varying partition: knots equal to the data at resolution 0."""
    locs, y = _data(40, 5)
    theta = (1.0, 0.3, 0.2)

    def knots(m, i, box):
        return locs if m == 0 else O.grid_knots(box, 4, 2)

    p = O.Problem(locs, y, M=2, J=(2, 8), family="exp", knots_fn=knots)
    assert O.loglik(p, theta) == pytest.approx(E.exact_loglik(locs, y, theta, "exp"), rel=1e-9)


def test_p4_bruteforce_differs_from_exact():
    """Control for P4: C_M is a genuine approximation on this tree."""
    locs, y = _data(220, 30)
    p = O.Problem(locs, y, M=2, r=4, family="exp")
    assert abs(E.bruteforce_loglik(p, TH_EXP) - E.exact_loglik(locs, y, TH_EXP, "exp")) > 1e-3


# ---- P5: C_M(s, s) = C0(s, s) (Sec. 2.4) ---------------------------------------

def test_p5_variance_invariant():
    locs, y = _data(150, 40)
    theta = (0.7, 0.2, 0.0)
    p = O.Problem(locs, y, M=3, r=4, family="matern15")
    CM = E.bruteforce_cov(p.tree, locs, theta[:2], "matern15")
    np.testing.assert_allclose(np.diag(CM), 0.7, rtol=1e-12)
    # and through the prior recursion: diag Sigma_leaf + sum_l diag B^l K_l B^l' = C0(s, s)
    P = O.prior(p.tree, locs, theta[:2], "matern15", 0.0)
    for f in range(4 ** 3):
        if p.tree.obs[f].size == 0:
            continue
        tot = np.diag(P.Sigma[f]).copy()
        for l, R in enumerate(O.ancestors(3, f, 4)[:3]):
            B = P.W[(3, f)][l]
            tot += np.sum((B @ P.K[R]) * B, axis=1)
        np.testing.assert_allclose(tot, 0.7, rtol=1e-11)


# ---- P6: M = 1 is the full-scale approximation (Sec. 2.4) -----------------------

def test_p6_one_level_full_scale_closed_form():
    locs, y = _data(120, 50)
    theta = (1.0, 0.25, 0.1)
    p = O.Problem(locs, y, M=1, r=9, family="exp")
    Q = p.tree.knots[0][0]
    C = E.c0(locs, locs, theta[:2], "exp")
    CQ = E.c0(locs, Q, theta[:2], "exp")
    low = CQ @ np.linalg.solve(E.c0(Q, Q, theta[:2], "exp"), CQ.T)
    cell = E.cell_index(locs, (0.0, 1.0, 0.0, 1.0), 4, 1, 2)   # the checker's own locator
    same = cell[:, None] == cell[None, :]
    C1 = low + np.where(same, C - low, 0.0)
    ll = E.gaussian_loglik(C1 + theta[2] * np.eye(120), y)
    assert O.loglik(p, theta) == pytest.approx(ll, rel=1e-12)


# ---- P7: Prop. 1 and posterior sanity -------------------------------------------

def test_p7_posterior_variance_bounds():
    locs, y = _data(300, 60)
    plocs, _ = _data(200, 61)
    theta = (1.0, 0.1, 0.05)
    p = O.Problem(locs, y, M=2, r=9, family="matern15")
    mu, var = O.predict(p, theta, plocs)
    assert np.all(var >= -1e-12)
    assert np.all(var <= 1.0 + 1e-12)


# ---- P8: gradient ---------------------------------------------------------------

@pytest.mark.parametrize("family", ["exp", "matern15"])
def test_p8_gradient_matches_central_differences(family):
    locs, y = _data(150, 70)
    theta = np.array(TH_M15 if family == "matern15" else TH_EXP)
    p = O.Problem(locs, y, M=2, r=9, family=family)
    _, g = O.loglik_grad(p, theta)
    h = 1e-5
    for a in range(3):
        tp, tm = theta.copy(), theta.copy()
        tp[a] *= 1 + h
        tm[a] *= 1 - h
        fd = (O.loglik(p, tp) - O.loglik(p, tm)) / (tp[a] - tm[a])
        assert g[a] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_p8_sigma2_closed_form_without_nugget():
    """With tau2 = 0, C_M is proportional to sigma2: d/dsigma2 = (u - n) / (2 sigma2)."""
    locs, y = _data(100, 80)
    theta = np.array([1.7, 0.2, 0.0])
    p = O.Problem(locs, y, M=2, r=4, family="exp")
    ll, g = O.loglik_grad(p, theta)
    _, _, Q = O.loglik(p, theta, return_state=True)
    u = Q.u[(0, 0)]
    assert g[0] == pytest.approx((u - 100) / (2 * 1.7), rel=1e-10)


def test_p8_scale_homogeneity():
    """Sigma(c sigma2, c tau2) = c Sigma: sigma2 g0 + tau2 g2 = (u - n) / 2."""
    locs, y = _data(100, 81)
    theta = np.array([0.8, 0.15, 0.07])
    p = O.Problem(locs, y, M=2, r=9, family="matern15")
    _, g = O.loglik_grad(p, theta)
    _, _, Q = O.loglik(p, theta, return_state=True)
    assert theta[0] * g[0] + theta[2] * g[2] == pytest.approx((Q.u[(0, 0)] - 100) / 2, rel=1e-10)


# ---- P9: invariances ------------------------------------------------------------

def test_p9_permutation_and_scaling():
    locs, y = _data(200, 90)
    theta = TH_EXP
    p = O.Problem(locs, y, M=2, r=9, family="exp")
    ll, _, Q = O.loglik(p, theta, return_state=True)
    perm = np.random.default_rng(1).permutation(200)
    pp = O.Problem(locs[perm], y[perm], M=2, r=9, family="exp")
    assert O.loglik(pp, theta) == pytest.approx(ll, rel=1e-12)
    c = 3.0
    _, _, Qc = O.loglik(O.Problem(locs, c * y, M=2, r=9, family="exp"), theta, return_state=True)
    assert Qc.d[(0, 0)] == pytest.approx(Q.d[(0, 0)], rel=1e-13)
    assert Qc.u[(0, 0)] == pytest.approx(c * c * Q.u[(0, 0)], rel=1e-12)


def test_empty_leaves_contribute_nothing():
    """Reading R10: data confined to one quadrant gives the same loglik as a tree
    whose other subtrees are absent."""
    rng = np.random.default_rng(100)
    locs = 0.5 * rng.random((90, 2))
    y = rng.standard_normal(90)
    theta = TH_EXP
    p = O.Problem(locs, y, M=3, r=4, family="exp")
    assert any(o.size == 0 for o in p.tree.obs)
    assert O.loglik(p, theta) == pytest.approx(E.bruteforce_loglik(p, theta), rel=1e-11)


def test_region_terms_add_up():
    """d_R, u_R of the children plus the parent's own update give the parent's."""
    locs, y = _data(200, 110)
    theta = TH_M15
    p = O.Problem(locs, y, M=2, r=4, family="matern15")
    _, _, Q = O.loglik(p, theta, return_state=True)
    for i in range(4):
        d, u = O.region_terms(p, theta, 1, i)
        assert d == pytest.approx(Q.d[(1, i)], rel=1e-12)
        assert u == pytest.approx(Q.u[(1, i)], rel=1e-12)


def test_not_positive_definite_is_reported():
    with pytest.raises(O.NotPositiveDefinite):
        O.chol(np.array([[1.0, 2.0], [2.0, 1.0]]))


# ---- P10: joint posterior predictive and conditional simulation (Prop. 2) ------

@pytest.mark.parametrize("M,r,family", [(1, 4, "exp"), (2, 9, "matern15"), (3, 4, "exp")])
def test_p10_joint_covariance_matches_bruteforce(M, r, family):
    """The covariance Prop. 2 implies between prediction points equals joint
    kriging under the dense C_M of the process definition; its diagonal is the
    marginal variance of predict."""
    locs, y = _data(200, 120 + M)
    rng = np.random.default_rng(121 + M)
    plocs = np.concatenate([rng.random((30, 2)), 0.26 + 0.02 * rng.random((6, 2))])   # a crowded leaf too
    theta = TH_M15 if family == "matern15" else TH_EXP
    p = O.Problem(locs, y, M=M, r=r, family=family)
    mean, cov = O.predict_joint(p, theta, plocs)
    mb, cb = E.bruteforce_predict_joint(p, theta, plocs)
    np.testing.assert_allclose(mean, mb, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(cov, cb, rtol=1e-8, atol=1e-10)
    mu, var = O.predict(p, theta, plocs)
    np.testing.assert_allclose(np.diag(cov), var, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(mean, mu, rtol=1e-10, atol=1e-12)
    assert np.allclose(cov, cov.T, rtol=0, atol=1e-12)


def test_p10_simulation_is_an_exact_linear_map():
    """A draw is mean + A [xi; zeta]: with xi, zeta = 0 it is the mean, and the
    map's columns (unit inputs) satisfy A A' = the joint covariance, i.e. the
    draws of standard normal inputs have exactly the predictive distribution."""
    locs, y = _data(150, 130)
    rng = np.random.default_rng(131)
    plocs = rng.random((12, 2))
    theta = TH_M15
    p = O.Problem(locs, y, M=2, r=4, family="matern15")
    _, P, Q = O.loglik(p, theta, return_state=True)
    mean, cov = O.predict_joint(p, theta, plocs, state=(P, Q))
    _, nxi = O.xi_offsets(p.tree)
    assert nxi == 4 * (1 + 4)
    npts = plocs.shape[0]
    zero = O.simulate(p, theta, plocs, np.zeros((1, nxi)), np.zeros((1, npts)), state=(P, Q))
    np.testing.assert_allclose(zero[0], mean, rtol=1e-12, atol=1e-14)
    eye = np.eye(nxi + npts)
    A = O.simulate(p, theta, plocs, eye[:, :nxi], eye[:, nxi:], state=(P, Q)) - mean
    np.testing.assert_allclose(A.T @ A, cov, rtol=1e-9, atol=1e-11)


# ---- P11: the Matern family of free smoothness (Sec. 4.1) -----------------------

TH_NU = (1.2, 0.15, 0.05, 2.3)


def test_p11_free_smoothness_exact_and_bruteforce():
    locs, y = _data(120, 150)
    plocs, _ = _data(10, 151)
    p0 = O.Problem(locs[:80], y[:80], M=0, r=4, family="matern")
    assert O.loglik(p0, TH_NU) == pytest.approx(E.exact_loglik(locs[:80], y[:80], TH_NU, "matern"), rel=1e-12)
    p = O.Problem(locs, y, M=2, r=9, family="matern")
    assert O.loglik(p, TH_NU) == pytest.approx(E.bruteforce_loglik(p, TH_NU), rel=1e-11)
    mu, var = O.predict(p, TH_NU, plocs)
    mb, vb = E.bruteforce_predict(p, TH_NU, plocs)
    np.testing.assert_allclose(mu, mb, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(var, vb, rtol=1e-8, atol=1e-10)
    # nu = 3/2 is Eq. mat15
    p15 = O.Problem(locs, y, M=2, r=9, family="matern15")
    assert O.loglik(p, (1.2, 0.15, 0.05, 1.5)) == pytest.approx(O.loglik(p15, (1.2, 0.15, 0.05)), rel=1e-12)


def test_p11_free_smoothness_gradient():
    locs, y = _data(150, 160)
    p = O.Problem(locs, y, M=2, r=9, family="matern")
    theta = np.array(TH_NU)
    _, g = O.loglik_grad(p, theta)
    assert g.shape == (4,)
    for a in range(4):
        tp, tm = theta.copy(), theta.copy()
        tp[a] *= 1 + 1e-5
        tm[a] *= 1 - 1e-5
        fd = (O.loglik(p, tp) - O.loglik(p, tm)) / (tp[a] - tm[a])
        assert g[a] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(g).max())
    _, _, Q = O.loglik(p, theta, return_state=True)
    assert theta[0] * g[0] + theta[2] * g[2] == pytest.approx((Q.u[(0, 0)] - 150) / 2, rel=1e-10)

"""Joint posterior predictive distribution and conditional simulation on the
GPU (Prop. 2) against the oracle.

The covariance between prediction points is compared element by element with
the oracle's (relative 1e-9 of its largest entry); draws from the same
standard normals are compared element by element (reading R17 fixes the square
roots both sides use); and the sample covariance of many seeded draws is
checked against the joint covariance (a moment check with a statistical bound).
"""
import numpy as np
import pytest

from oracle import mra_oracle as O

pytestmark = pytest.mark.gpu

RTOL = 1e-9


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


def _problem(seed, n, M, r, family, npred):
    rng = np.random.default_rng(seed)
    locs = rng.random((n, 2))
    y = rng.standard_normal(n)
    plocs = np.concatenate([rng.random((npred, 2)), 0.3 + 0.01 * rng.random((5, 2))])   # one crowded leaf
    return locs, y, plocs


@pytest.mark.parametrize("M,r,family,precision", [(2, 16, "exp", "fp64"), (3, 9, "matern15", "fp64"),
                                                  (3, 16, "matern15", "emu"), (0, 4, "exp", "fp64")])
def test_joint_covariance_matches_oracle(mra, M, r, family, precision):
    locs, y, plocs = _problem(40 + M, 900 if M else 120, M, r, family, 120 if M else 40)   # M = 0: one leaf
    theta = (1.2, 0.15, 0.04)
    p = O.Problem(locs, y, M=M, r=r, family=family)
    mo, co = O.predict_joint(p, theta, plocs)
    with mra.Handle(locs, y, M=M, r=r, family=family, precision=precision) as h:
        mg, cg = h.predict_joint(theta, plocs)
        mm, vm = h.predict(theta, plocs)
    scale = np.abs(co).max()
    np.testing.assert_allclose(cg, co, rtol=RTOL, atol=RTOL * scale)
    np.testing.assert_allclose(mg, mo, rtol=RTOL, atol=RTOL * np.abs(mo).max())
    np.testing.assert_allclose(np.diag(cg), vm, rtol=1e-12, atol=1e-14 * scale)   # the marginal kernel agrees
    np.testing.assert_allclose(mg, mm, rtol=1e-12, atol=1e-14)


def test_simulation_matches_oracle_draw_by_draw(mra):
    locs, y, plocs = _problem(50, 1200, 3, 16, "matern15", 80)
    theta = (1.0, 0.12, 0.03)
    p = O.Problem(locs, y, M=3, r=16, family="matern15")
    rng = np.random.default_rng(51)
    with mra.Handle(locs, y, M=3, r=16, family="matern15") as h:
        nxi = h.xi_len()
        assert nxi == 16 * (1 + 4 + 16)
        xi = rng.standard_normal((7, nxi))
        zeta = rng.standard_normal((7, plocs.shape[0]))
        dg = h.simulate(theta, plocs, xi, zeta)
        zero = h.simulate(theta, plocs, np.zeros((1, nxi)), np.zeros((1, plocs.shape[0])))
        mg, _ = h.predict(theta, plocs)
    do = O.simulate(p, theta, plocs, xi, zeta)
    np.testing.assert_allclose(dg, do, rtol=RTOL, atol=RTOL * np.abs(do).max())
    np.testing.assert_allclose(zero[0], mg, rtol=1e-12, atol=1e-13)


def test_simulation_moments_and_device_buffers(mra):
    torch = pytest.importorskip("torch")
    locs, y, plocs = _problem(60, 1500, 2, 16, "exp", 40)
    theta = (1.0, 0.2, 0.05)
    nsim = 20000
    with mra.Handle(locs, y, M=2, r=16, family="exp") as h:
        mean, cov = h.predict_joint(theta, plocs)
        g = torch.Generator(device="cuda").manual_seed(61)
        xi = torch.randn((nsim, h.xi_len()), generator=g, device="cuda", dtype=torch.float64)
        zeta = torch.randn((nsim, plocs.shape[0]), generator=g, device="cuda", dtype=torch.float64)
        dp = torch.tensor(plocs, device="cuda")
        draws = h.simulate(theta, dp, xi, zeta).cpu().numpy()
        md, cd = h.predict_joint(theta, dp)
    np.testing.assert_array_equal(md.cpu().numpy(), mean)
    np.testing.assert_array_equal(cd.cpu().numpy(), cov)
    sd = np.sqrt(np.diag(cov))
    emp_mean = draws.mean(axis=0)
    emp_cov = np.cov(draws, rowvar=False)
    # standard errors: mean sd / sqrt(nsim); covariance about (sd_i sd_j) sqrt(2 / nsim)
    assert np.all(np.abs(emp_mean - mean) <= 5 * sd / np.sqrt(nsim))
    assert np.all(np.abs(emp_cov - cov) <= 6 * np.outer(sd, sd) * np.sqrt(2.0 / nsim))


def test_joint_limits(mra):
    rng = np.random.default_rng(70)
    locs = rng.random((500, 2))
    y = rng.standard_normal(500)
    with mra.Handle(locs, y, M=2, r=16) as h:
        crowded = 0.1 * rng.random((70, 2))              # 70 points in one leaf
        with pytest.raises(mra.MRAError) as ei:
            h.predict_joint((1.0, 0.1, 0.01), crowded)
        assert ei.value.code == mra.MRA_ERR_LIMIT
        with pytest.raises(ValueError):
            h.simulate((1.0, 0.1, 0.01), rng.random((3, 2)), np.zeros((1, h.xi_len() + 1)), np.zeros((1, 3)))

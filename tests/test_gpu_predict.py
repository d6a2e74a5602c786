"""GPU kriging parity with the FP64 oracle (Sec. 3.4, Prop. 2).

Posterior predictive means and variances of y at prediction points, element by
element against the oracle's Prop. 2 (definition at l = M, recursion below),
to a relative 1e-9.  Cases: the n = 4096 workload with its 1024 points, several
tree shapes, points in empty leaves, more points in one leaf than one CTA takes,
host and device buffers.
"""
import numpy as np
import pytest

from oracle import mra_oracle as O
from paper_1507_04789_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-9


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


def _check(mra, locs, y, plocs, M, r, family, theta, nonstat=False):
    p = O.Problem(locs, y, M=M, r=r, family=family, nonstat=nonstat)
    mo, vo = O.predict(p, theta, plocs)
    with mra.Handle(locs, y, M=M, r=r, family=family, nonstat=nonstat) as h:
        h.loglik(theta)
        mg, vg = h.predict(theta, plocs)
    scale_m = np.abs(mo).max() + 1e-300
    np.testing.assert_allclose(mg, mo, rtol=RTOL, atol=RTOL * scale_m)
    np.testing.assert_allclose(vg, vo, rtol=RTOL, atol=RTOL * theta[0] * 1e-3)
    return mg, vg


def test_n4096_exponential_1024_points(mra):
    w = synth.workload("n4096_exp_M3_r16")
    locs, y, plocs = w.generate()
    _check(mra, locs, y, plocs, w.M, w.r, w.family, (w.sigma2, w.kappa, w.tau2))


@pytest.mark.parametrize("n,M,r,family,nonstat,npred,seed", [
    (300, 2, 9, "exp", False, 200, 1),
    (800, 2, 64, "matern15", False, 300, 2),
    (100, 0, 16, "matern15", False, 50, 3),
    (600, 3, 16, "exp", True, 400, 4),
    (1200, 3, 36, "matern15", False, 500, 5),
])
def test_parity_grid(mra, n, M, r, family, nonstat, npred, seed):
    rng = np.random.default_rng(seed)
    locs = rng.random((n, 2))
    y = rng.standard_normal(n)
    plocs = rng.random((npred, 2))
    theta = (1.3, 0.1, 0.02) if family == "matern15" else (0.8, 0.25, 0.1)
    _check(mra, locs, y, plocs, M, r, family, theta, nonstat)


def test_empty_leaves_and_crowded_leaf(mra):
    """Data in one quadrant; 300 prediction points in a single leaf (several CTAs)."""
    rng = np.random.default_rng(6)
    locs = 0.5 * rng.random((380, 2))                   # about 95 per non-empty leaf
    y = rng.standard_normal(380)
    crowd = 0.6 + 0.1 * rng.random((300, 2))            # one empty leaf at M = 2
    spread = rng.random((150, 2))
    plocs = np.concatenate([crowd, spread])
    _check(mra, locs, y, plocs, 2, 16, "exp", (1.0, 0.2, 0.05))


def test_prediction_at_observed_locations(mra):
    """Variance of y at an observed location is below tau2-free prior variance."""
    rng = np.random.default_rng(7)
    locs = rng.random((400, 2))
    y = rng.standard_normal(400)
    mg, vg = _check(mra, locs, y, locs[:50], 2, 16, "matern15", (1.0, 0.1, 0.05))
    assert np.all(vg > 0) and np.all(vg < 1.0)


def test_device_buffers_and_state(mra):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    locs = rng.random((700, 2))
    y = rng.standard_normal(700)
    plocs = rng.random((120, 2))
    theta = (1.0, 0.15, 0.03)
    with mra.Handle(locs, y, M=2, r=16) as h:
        m_first, v_first = h.predict(theta, plocs)       # no evaluation yet: the call evaluates at theta
        ll = h.loglik(theta)
        m_host, v_host = h.predict(theta, plocs)
        np.testing.assert_array_equal(m_first, m_host)
        np.testing.assert_array_equal(v_first, v_host)
        m_dev, v_dev = h.predict(theta, torch.tensor(plocs, device="cuda"))
        np.testing.assert_array_equal(m_dev.cpu().numpy(), m_host)
        np.testing.assert_array_equal(v_dev.cpu().numpy(), v_host)
        theta2 = (1.0, 0.2, 0.03)                        # another theta: evaluated first, then predicted
        m2, v2 = h.predict(theta2, plocs)
        p = O.Problem(locs, y, M=2, r=16, family="exp")
        mo, vo = O.predict(p, theta2, plocs)
        np.testing.assert_allclose(m2, mo, rtol=RTOL, atol=RTOL)
        np.testing.assert_allclose(v2, vo, rtol=RTOL, atol=RTOL)
        assert h.region_terms(0)[0][0] == pytest.approx(O.region_terms(p, theta2, 0, 0)[0], rel=1e-10)
        with pytest.raises(mra.MRAError) as ei:
            h.predict((1.0, -0.2, 0.03), plocs)
        assert ei.value.code == mra.MRA_ERR_ARG
        h.predict(theta, plocs)
        assert h.loglik(theta) == ll
        big = rng.random((5000, 2))                      # grows the prediction buffer
        mb, vb = h.predict(theta, big)
        np.testing.assert_array_equal(h.predict(theta, plocs)[0], m_host)


@pytest.mark.parametrize("r,M", [(64, 3), (16, 3), (32, 3)])
def test_sparse_points_take_the_short_tile(mra, r, M):
    """At most 16 points per leaf run in 16-row tiles (the n = 2^24 grid has about
    one point per leaf): the same points give the same means and variances,
    bitwise, as inside a crowded set that takes the full tiles, and the oracle's."""
    rng = np.random.default_rng(2 + r)
    n = 3000
    locs = rng.random((n, 2))
    y = rng.standard_normal(n)
    theta = (1.0, 0.2, 0.05)
    sparse = rng.random((60, 2))                  # 64 leaves at M = 3: about one point per leaf
    crowded = np.concatenate([sparse, rng.random((4000, 2))])
    with mra.Handle(locs, y, M=M, r=r, family="matern15") as h:
        h.loglik(theta)
        m1, v1 = h.predict(theta, sparse)
        m2, v2 = h.predict(theta, crowded)
    np.testing.assert_array_equal(m1, m2[:60])
    np.testing.assert_array_equal(v1, v2[:60])
    p = O.Problem(locs, y, M=M, r=r, family="matern15")
    mo, vo = O.predict(p, theta, sparse)
    np.testing.assert_allclose(m1, mo, rtol=RTOL, atol=RTOL * np.abs(mo).max())
    np.testing.assert_allclose(v1, vo, rtol=RTOL, atol=RTOL * theta[0] * 1e-3)

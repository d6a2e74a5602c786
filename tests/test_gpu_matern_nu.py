"""The Matern family of free smoothness nu (MRA_COV_MATERN) on the GPU against
the oracle: log-likelihood (1e-10), predictions (1e-9) and the four-component
gradient, whose d/dnu comes from the hand-written adjoint on the GPU and from
extrapolated central differences in the oracle (1e-6 there, 1e-8 for the
complex-step components)."""
import numpy as np
import pytest

from oracle import mra_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


def _data(seed, n=1500):
    rng = np.random.default_rng(seed)
    return rng.random((n, 2)), rng.standard_normal(n), rng.random((60, 2))


@pytest.mark.parametrize("nu,precision", [(0.8, "fp64"), (2.3, "fp64"), (2.3, "emu")])
def test_loglik_and_prediction(mra, nu, precision):
    locs, y, plocs = _data(170)
    theta = (1.1, 0.12, 0.04, nu)
    p = O.Problem(locs, y, M=3, r=16, family="matern")
    ll_o = O.loglik(p, theta)
    mo, vo = O.predict(p, theta, plocs)
    with mra.Handle(locs, y, M=3, r=16, family="matern", precision=precision) as h:
        assert h.loglik(theta) == pytest.approx(ll_o, rel=1e-10)
        mg, vg = h.predict(theta, plocs)
    np.testing.assert_allclose(mg, mo, rtol=1e-9, atol=1e-9 * np.abs(mo).max())
    np.testing.assert_allclose(vg, vo, rtol=1e-9, atol=1e-12)


def test_half_integer_smoothness_equals_closed_form(mra):
    locs, y, _ = _data(171)
    with mra.Handle(locs, y, M=3, r=16, family="matern") as h, mra.Handle(locs, y, M=3, r=16, family="matern15") as h15:
        assert h.loglik((1.0, 0.1, 0.02, 1.5)) == pytest.approx(h15.loglik((1.0, 0.1, 0.02)), rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_four_component_gradient(mra, precision):
    locs, y, _ = _data(172, n=1200)
    theta = np.array([1.1, 0.12, 0.04, 1.9])
    p = O.Problem(locs, y, M=3, r=16, family="matern")
    ll_o, g_o = O.loglik_grad(p, theta)
    with mra.Handle(locs, y, M=3, r=16, family="matern", precision=precision) as h:
        ll, g = h.loglik_grad(theta)
    assert g.shape == (4,)
    assert ll == pytest.approx(ll_o, rel=1e-10)
    scale = np.abs(g_o[:3]).max()
    np.testing.assert_allclose(g[:3], g_o[:3], rtol=1e-8, atol=1e-8 * scale)
    assert g[3] == pytest.approx(g_o[3], rel=1e-6, abs=1e-6 * scale)

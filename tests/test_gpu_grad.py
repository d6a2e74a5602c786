"""GPU gradient of the log-likelihood against the oracle.

The GPU gradient is the reverse-mode adjoint of the FP64 evaluation; the
oracle's is the complex-step derivative of its own loglik (exact to rounding).
They must agree to a relative 1e-8 per component (relative to the largest
component, so that a near-zero component is judged on the gradient's scale).
Central differences of the GPU loglik and the scale-homogeneity identity
sigma2 g_sigma2 + tau2 g_tau2 = (u - n)/2 are checked as well.
"""
import numpy as np
import pytest

from oracle import mra_oracle as O
from paper_1507_04789_gb300 import synth

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-8


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


def _cmp(g, go, rtol=GRAD_RTOL):
    scale = np.abs(go).max()
    np.testing.assert_allclose(g, go, rtol=rtol, atol=rtol * scale)


@pytest.mark.parametrize("n,M,r,family,nonstat,seed", [
    (200, 0, 16, "exp", False, 1),
    (300, 1, 9, "exp", False, 2),
    (400, 2, 16, "matern15", False, 3),
    (600, 3, 4, "exp", True, 4),
    (900, 2, 64, "matern15", False, 5),
    (1500, 3, 25, "matern15", False, 6),
])
def test_gradient_matches_oracle(mra, n, M, r, family, nonstat, seed):
    rng = np.random.default_rng(seed)
    locs = rng.random((n, 2))
    if M == 0:
        locs = locs[:100]
        n = 100
    y = rng.standard_normal(n)
    theta = np.array([1.3, 0.12, 0.04]) if family == "matern15" else np.array([0.8, 0.2, 0.07])
    p = O.Problem(locs, y, M=M, r=r, family=family, nonstat=nonstat)
    ll_o, g_o = O.loglik_grad(p, theta)
    with mra.Handle(locs, y, M=M, r=r, family=family, nonstat=nonstat) as h:
        ll, g = h.loglik_grad(theta)
        assert ll == pytest.approx(ll_o, rel=1e-10)
        _cmp(g, g_o)
        assert h.loglik(theta) == ll                       # same forward


def test_gradient_n4096_workload(mra):
    w = synth.workload("n4096_exp_M3_r16")
    locs, y, _ = w.generate()
    theta = np.array([w.sigma2, w.kappa, w.tau2])
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    _, g_o = O.loglik_grad(p, theta)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family) as h:
        _, g = h.loglik_grad(theta)
    _cmp(g, g_o)


def test_gradient_n16k_matern_M4_r64(mra):
    """2^14 points, the leaf shape of the 2^20 workload (M = 4, r = 64)."""
    w = synth.workload("n16k_matern15_M4_r64")
    locs, y, _ = w.generate()
    theta = np.array([w.sigma2, w.kappa, w.tau2])
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    _, g_o = O.loglik_grad(p, theta)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family) as h:
        _, g = h.loglik_grad(theta)
    _cmp(g, g_o)


def test_central_differences_and_homogeneity(mra):
    rng = np.random.default_rng(7)
    locs = rng.random((1200, 2))
    y = rng.standard_normal(1200)
    theta = np.array([1.1, 0.15, 0.05])
    with mra.Handle(locs, y, M=3, r=16, family="matern15") as h:
        ll, g = h.loglik_grad(theta)
        _, u0 = h.region_terms(0)
        for a in range(3):
            tp, tm = theta.copy(), theta.copy()
            tp[a] *= 1 + 1e-5
            tm[a] *= 1 - 1e-5
            fd = (h.loglik(tp) - h.loglik(tm)) / (tp[a] - tm[a])
            assert g[a] == pytest.approx(fd, rel=1e-5, abs=1e-5 * np.abs(g).max())
    assert theta[0] * g[0] + theta[2] * g[2] == pytest.approx((u0[0] - 1200) / 2, rel=1e-9)


def test_gradient_then_predict(mra):
    rng = np.random.default_rng(8)
    locs = rng.random((500, 2))
    y = rng.standard_normal(500)
    plocs = rng.random((40, 2))
    theta = (1.0, 0.2, 0.05)
    with mra.Handle(locs, y, M=2, r=16) as h:
        h.loglik(theta)
        m1, v1 = h.predict(theta, plocs)
        h.loglik_grad(theta)
        m2, v2 = h.predict(theta, plocs)
    np.testing.assert_array_equal(m1, m2)
    np.testing.assert_array_equal(v1, v2)


def test_autograd_function_and_mle(mra):
    """torch.autograd path and 20 steps of gradient-based MLE from range = 0.3."""
    torch = pytest.importorskip("torch")
    from paper_1507_04789_gb300 import autograd as ag
    w = synth.workload("n4096_exp_M3_r16")
    locs, y, _ = w.generate()
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family) as h:
        theta = torch.tensor([1.0, 0.3, 0.05], dtype=torch.float64, requires_grad=True)
        ll = ag.loglik(h, theta)
        ll.backward()
        _, g = h.loglik_grad(theta.detach().numpy())
        np.testing.assert_allclose(theta.grad.numpy(), g, rtol=0, atol=0)
        th, hist = ag.fit_mle(h, (1.0, 0.3, 0.05), steps=20, lr=0.1)
    lls = [v for _, v in hist]
    assert lls[-1] > lls[0] + 1.0            # the fit climbs the likelihood
    assert th[1] < 0.3                       # towards the generating range 0.05

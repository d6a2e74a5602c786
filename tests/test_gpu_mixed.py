"""Mixed-precision form (tensor-core 3xTF32 prior/leaf contractions) against the FP64 oracle.

The stated error bound of the mixed form is |d loglik| / n <= 1e-6 (the
FP64 form is held to a relative 1e-10).  Predictions and the gradient computed
from the mixed factors are held to bounds derived from the same arithmetic:
products with relative error near 2^-22 (3xTF32), accumulated in FP64.
"""
import numpy as np
import pytest

from oracle import mra_oracle as O
from paper_1507_04789_gb300 import synth

pytestmark = pytest.mark.gpu

LL_PER_OBS = 1e-6


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


@pytest.mark.parametrize("name", ["n4096_exp_M3_r16", "n16k_matern15_M4_r64"])
def test_mixed_loglik_within_bound(mra, name):
    w = synth.workload(name)
    locs, y, plocs = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    ll_o = O.loglik(p, theta)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision="mixed") as h:
        ll = h.loglik(theta)
        err = abs(ll - ll_o) / w.n
        print(f"{name}: mixed loglik {ll:.10f} oracle {ll_o:.10f} |d|/n = {err:.3e}")
        assert err <= LL_PER_OBS
        mean, var = h.predict(theta, plocs[:256])
    mo, vo = O.predict(p, theta, plocs[:256])
    em = np.abs(mean - mo).max() / np.abs(mo).max()
    ev = np.abs(var - vo).max() / np.abs(vo).max()
    print(f"{name}: prediction max rel err mean {em:.3e} var {ev:.3e}")
    assert em <= 1e-4 and ev <= 1e-4


def test_mixed_gradient(mra):
    w = synth.workload("n4096_exp_M3_r16")
    locs, y, _ = w.generate()
    theta = np.array([w.sigma2, w.kappa, w.tau2])
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    _, g_o = O.loglik_grad(p, theta)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision="mixed") as h:
        _, g = h.loglik_grad(theta)
    rel = np.abs(g - g_o).max() / np.abs(g_o).max()
    print(f"mixed gradient max rel err {rel:.3e}")
    assert rel <= 1e-4


def test_mixed_matches_fp64_on_gpu(mra):
    """GP-like data (the bound is relative to u = y' Sigma^{-1} y, about n for such data)."""
    locs = synth.uniform_locations(3000, 3)
    y = synth.noisy_observations(synth.rff_field(locs, 1.5, 0.1, 1.2, 4), 0.02, 5)
    theta = (1.2, 0.1, 0.02)
    with mra.Handle(locs, y, M=3, r=64, family="matern15") as h64, \
            mra.Handle(locs, y, M=3, r=64, family="matern15", precision="mixed") as hm:
        a, b = h64.loglik(theta), hm.loglik(theta)
        assert abs(a - b) / 3000 <= LL_PER_OBS
        d64, u64 = h64.region_terms(3)
        dm, um = hm.region_terms(3)
        np.testing.assert_allclose(dm, d64, rtol=1e-5, atol=1e-6 * np.abs(d64).max())
        assert hm.loglik(theta) == b                       # deterministic

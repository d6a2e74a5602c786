"""The headline workload itself against the oracle: n = 2^20 uniform points,
Matern-1.5 (sigma2 = 1, range 0.1, tau2 = 0.01), M = 7, r = 64, seed 0 (the
problem bench.py times).  The oracle evaluates two level-2 subtrees of it (each
1/16 of the leaves, a few seconds); their region terms d_R, u_R (Sec. 3.3)
must match the GPU's at a relative 1e-10 in the FP64 form and 5e-10 in the
emulated form: its products carry about 1e-14 relative to sum |a b|, the prior
chain C - V V' cancels by 1e4-1e5 at the finest levels, and u_R = sum of the
children's u - g'g loses further digits to that subtraction (measured 1.4e-10
here and up to 2.1e-10 on level-3 regions, while the root log-likelihood stays
within 2e-12 per observation of the FP64 form's).  Also the emulated leaf
kernels at the 128-observation maximum against the oracle."""
import numpy as np
import pytest

from oracle import mra_oracle as O
from paper_1507_04789_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


def test_headline_workload_region_terms(mra):
    w = synth.workload("n1M_matern15_M7_r64")
    locs, y, _ = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    regions = (5, 10)
    ref = [O.region_terms(p, theta, 2, k) for k in regions]
    for precision in ("fp64", "emu"):
        with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision) as h:
            h.loglik(theta)
            d, u = h.region_terms(2)
        tol = 1e-10 if precision == "fp64" else 5e-10
        for k, (do, uo) in zip(regions, ref):
            assert d[k] == pytest.approx(do, rel=tol), (precision, k)
            assert u[k] == pytest.approx(uo, rel=tol), (precision, k)


def test_emulated_full_leaves(mra):
    """Every leaf holds the 128-observation maximum (M = 3, 64 leaves, r = 16),
    and a second dataset mixes full, ragged and empty leaves."""
    rng = np.random.default_rng(180)
    cells = [(i, j) for j in range(8) for i in range(8)]
    locs = np.concatenate([(np.array(c) + rng.random((128, 2))) / 8.0 for c in cells])
    y = synth.noisy_observations(synth.rff_field(locs, 1.5, 0.1, 1.0, 181, 256), 0.02, 182)
    theta = (1.0, 0.1, 0.02)
    for family in ("exp", "matern15"):
        p = O.Problem(locs, y, M=3, r=16, family=family)
        with mra.Handle(locs, y, M=3, r=16, family=family, precision="emu") as h:
            assert np.diff(h.leaf_offsets()).max() == 128
            assert h.loglik(theta) == pytest.approx(O.loglik(p, theta), rel=1e-10)
            ll_g, g = h.loglik_grad(theta)
        _, g_o = O.loglik_grad(p, theta)
        np.testing.assert_allclose(g, g_o, rtol=1e-8, atol=1e-8 * np.abs(g_o).max())

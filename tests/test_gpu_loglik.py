"""GPU log-likelihood parity with the FP64 oracle (Sec. 3.1-3.3).

Element by element on the same seeded inputs: the log-likelihood to a relative
1e-10 and the per-region log-determinants d_R and quadratic forms u_R of every
level (basis-independent, so the whitened GPU form and the paper's K-form must
agree).  Cases span several tiles, ragged and empty leaves, every covariance
family and knot count up to r = 64.
"""
import math

import numpy as np
import pytest

from oracle import mra_oracle as O
from paper_1507_04789_gb300 import synth

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-10


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


def _problem(n, seed, clustered=False):
    rng = np.random.default_rng(seed)
    if clustered:   # uneven occupancy: most points in one quadrant, some leaves empty
        locs = np.concatenate([0.45 * rng.random((n - n // 5, 2)), rng.random((n // 5, 2))])
    else:
        locs = rng.random((n, 2))
    y = rng.standard_normal(n)
    return locs, y


def _compare(mra, locs, y, M, r, family, theta, nonstat=False, terms=True):
    p = O.Problem(locs, y, M=M, r=r, family=family, nonstat=nonstat)
    ll_o, _, Q = O.loglik(p, theta, return_state=True)
    with mra.Handle(locs, y, M=M, r=r, family=family, nonstat=nonstat) as h:
        ll_g = h.loglik(theta)
        assert ll_g == pytest.approx(ll_o, rel=LL_RTOL, abs=0)
        if terms:
            scale = abs(Q.d[(0, 0)]) + abs(Q.u[(0, 0)]) + 1.0
            for m in range(M + 1):
                d_g, u_g = h.region_terms(m)
                d_o = np.array([Q.d.get((m, i), 0.0) for i in range(4 ** m)])
                u_o = np.array([Q.u.get((m, i), 0.0) for i in range(4 ** m)])
                np.testing.assert_allclose(d_g, d_o, rtol=1e-10, atol=1e-11 * scale)
                np.testing.assert_allclose(u_g, u_o, rtol=1e-10, atol=1e-11 * scale)
    return ll_g, ll_o


def test_n4096_exponential_M3_r16(mra):
    """4096 uniform points, exponential (1, 0.05), tau2 = 0.05, M = 3, r = 16."""
    w = synth.workload("n4096_exp_M3_r16")
    locs, y, _ = w.generate()
    _compare(mra, locs, y, w.M, w.r, w.family, (w.sigma2, w.kappa, w.tau2))


@pytest.mark.parametrize("n,M,r,family,nonstat,clustered,seed", [
    (300, 2, 9, "exp", False, False, 1),
    (500, 3, 4, "matern15", True, False, 2),
    (900, 2, 64, "matern15", False, False, 3),
    (400, 1, 32, "exp", False, False, 4),
    (100, 0, 16, "exp", False, False, 5),
    (700, 3, 16, "exp", False, True, 6),
    (1500, 4, 25, "matern15", False, True, 7),
    (1500, 3, 49, "exp", True, True, 10),
    (2500, 3, 36, "matern15", False, False, 8),
])
def test_parity_grid(mra, n, M, r, family, nonstat, clustered, seed):
    locs, y = _problem(n, seed, clustered)
    theta = (1.2, 0.12, 0.03) if family == "matern15" else (0.9, 0.2, 0.08)
    _compare(mra, locs, y, M, r, family, theta, nonstat)


def test_ragged_full_leaves(mra):
    """Leaves from 0 up to the 128-observation maximum, several row tiles."""
    rng = np.random.default_rng(9)
    q = 0.5 * rng.random((255, 2))
    parts = [q[:128], q[128:165] + [0.5, 0.0], q[165:] + [0.5, 0.5]]   # leaves of 128, 37, 0, 90
    locs = np.concatenate(parts)
    y = rng.standard_normal(locs.shape[0])
    with mra.Handle(locs, y, M=1, r=16) as h:
        off = h.leaf_offsets()
    np.testing.assert_array_equal(np.diff(off), [128, 37, 0, 90])
    _compare(mra, locs, y, 1, 16, "exp", (1.0, 0.3, 0.1))


def test_set_data_and_repeat(mra):
    locs, y = _problem(600, 11)
    y2 = np.random.default_rng(12).standard_normal(600)
    theta = (1.0, 0.15, 0.05)
    p2 = O.Problem(locs, y2, M=2, r=16, family="exp")
    with mra.Handle(locs, y, M=2, r=16) as h:
        a = h.loglik(theta)
        assert h.loglik(theta) == a                   # deterministic
        h.set_data(y2)
        assert h.loglik(theta) == pytest.approx(O.loglik(p2, theta), rel=LL_RTOL)


def test_device_inputs(mra):
    torch = pytest.importorskip("torch")
    locs, y = _problem(800, 13)
    theta = (1.0, 0.1, 0.02)
    with mra.Handle(locs, y, M=2, r=16, family="matern15") as h:
        ref = h.loglik(theta)
    dl = torch.tensor(locs, device="cuda")
    dy = torch.tensor(y, device="cuda")
    with mra.Handle(dl, dy, M=2, r=16, family="matern15") as h:
        assert h.loglik(theta) == ref


def test_sorted_order_is_stable(mra):
    locs, y = _problem(1000, 14)
    with mra.Handle(locs, y, M=3, r=4) as h:
        off, perm = h.leaf_offsets(with_perm=True)
    tree = O.build_tree(locs, 3, 4, 4)
    for f in range(64):
        np.testing.assert_array_equal(perm[off[f]:off[f + 1]], tree.obs[f])


def test_errors(mra):
    rng = np.random.default_rng(15)
    locs = rng.random((50, 2))
    y = rng.standard_normal(50)
    with pytest.raises(mra.MRAError) as ei:
        bad = locs.copy()
        bad[3, 0] = 1.5
        mra.Handle(bad, y, M=1, r=4)
    assert ei.value.code == mra.MRA_ERR_ARG
    with pytest.raises(mra.MRAError) as ei:
        mra.Handle(rng.random((200, 2)), rng.standard_normal(200), M=0, r=4)
    assert ei.value.code == mra.MRA_ERR_LIMIT
    dup = np.concatenate([locs, locs[:5]])
    with mra.Handle(dup, rng.standard_normal(55), M=1, r=4) as h:
        with pytest.raises(mra.MRAError) as ei:
            h.loglik((1.0, 0.2, 0.0))                 # duplicate points, no nugget
        assert ei.value.code == mra.MRA_ERR_NOT_PD
        assert math.isfinite(h.loglik((1.0, 0.2, 0.1)))   # recovers with a nugget
        with pytest.raises(mra.MRAError) as ei:
            h.loglik((1.0, -0.2, 0.1))
        assert ei.value.code == mra.MRA_ERR_ARG

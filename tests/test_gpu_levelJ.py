"""GPU parity on partitions with level-varying J (Sec. 2.2; Sec. 4.3 varies J_m).

Every level-(m-1) region splits into an s_x x s_y grid of equal children by
repeated midpoint halving (J_m = s_x s_y in {2, 4, 8, 16}, the halvings
alternating x, y over the whole sequence).  Against the FP64 oracle on the same
seeded inputs: the partition bit-exact (leaf offsets and in-leaf order), the
log-likelihood and every level's d_R, u_R, the gradient, kriging means and
variances and the joint predictive covariance, in the three precision forms, on
complete and pruned trees, streamed, and in a batch of mixed partitions.
"""
import numpy as np
import pytest

from oracle import mra_oracle as O

pytestmark = pytest.mark.gpu

TH_EXP = (0.9, 0.15, 0.05)
TH_M15 = (1.2, 0.12, 0.03)


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


def _data(n, seed, clustered=False):
    rng = np.random.default_rng(seed)
    locs = rng.random((n, 2))
    if clustered:   # uneven occupancy and empty leaves: the upper right corner moved to the centre
        hole = (locs[:, 0] > 0.55) & (locs[:, 1] > 0.55)
        locs[hole] *= 0.6
    return locs, rng.standard_normal(n)


def _theta(family):
    return TH_M15 if family == "matern15" else TH_EXP


def _ll_tol(precision, n):
    # 3xTF32 keeps about 1e-6 of the log-likelihood per observation (the form's
    # stated bound on the n = 2^20 workload); this n = 1500 exponential case
    # measured 1.02e-6, so the test allows twice the bound
    return 2e-6 * n if precision == "mixed" else None


CASES = [   # J, r, family, precision, prune, n, clustered
    ((8, 2), 16, "exp", "fp64", False, 1200, False),
    ((2, 8, 4), 16, "matern15", "emu", True, 1800, True),
    ((8, 2, 4), 9, "exp", "mixed", False, 1500, False),
    ((16, 4), 16, "exp", "emu", False, 2000, False),
    ((4, 16, 2), 16, "matern15", "fp64", True, 2500, True),
    ((2, 2, 4, 4), 64, "matern15", "emu", False, 4000, False),
]


@pytest.mark.parametrize("J,r,family,precision,prune,n,clustered", CASES)
def test_loglik_and_region_terms(mra, J, r, family, precision, prune, n, clustered):
    locs, y = _data(n, 7 + sum(J) + r, clustered)
    M = len(J)
    theta = _theta(family)
    p = O.Problem(locs, y, M=M, J=J, r=r, family=family)
    ll_o, _, Q = O.loglik(p, theta, return_state=True)
    with mra.Handle(locs, y, M=M, r=r, J=J, family=family, precision=precision, prune=prune) as h:
        off, perm = h.leaf_offsets(with_perm=True)     # the partition, bit-exact
        tree = p.tree
        assert off.shape[0] == tree.nreg(M) + 1
        for i in range(tree.nreg(M)):
            np.testing.assert_array_equal(perm[off[i]:off[i + 1]], tree.obs[i])
        ll = h.loglik(theta)
        if precision == "mixed":
            assert abs(ll - ll_o) <= _ll_tol(precision, n)
            return
        assert ll == pytest.approx(ll_o, rel=1e-10)
        scale = abs(Q.d[(0, 0)]) + abs(Q.u[(0, 0)]) + 1.0
        for m in range(M + 1):
            d_g, u_g = h.region_terms(m)
            assert d_g.shape[0] == tree.nreg(m)
            d_o = np.array([Q.d.get((m, i), 0.0) for i in range(tree.nreg(m))])
            u_o = np.array([Q.u.get((m, i), 0.0) for i in range(tree.nreg(m))])
            np.testing.assert_allclose(d_g, d_o, rtol=1e-10, atol=1e-11 * scale)
            np.testing.assert_allclose(u_g, u_o, rtol=1e-10, atol=1e-11 * scale)


@pytest.mark.parametrize("J,r,family,precision", [((8, 2), 16, "exp", "fp64"), ((8, 2, 4), 9, "matern15", "emu"),
                                                  ((16, 4), 16, "exp", "emu")])
def test_gradient(mra, J, r, family, precision):
    locs, y = _data(1200, 30 + sum(J))
    M = len(J)
    theta = np.array(_theta(family))
    ll_o, g_o = O.loglik_grad(O.Problem(locs, y, M=M, J=J, r=r, family=family), theta)
    with mra.Handle(locs, y, M=M, r=r, J=J, family=family, precision=precision) as h:
        ll, g = h.loglik_grad(theta)
    assert ll == pytest.approx(ll_o, rel=1e-10)
    scale = np.abs(g_o).max()
    np.testing.assert_allclose(g, g_o, rtol=1e-8, atol=1e-8 * scale)


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_prediction_and_joint_covariance(mra, precision):
    J, r, family = (2, 8, 2), 16, "matern15"
    locs, y = _data(1500, 41)
    rng = np.random.default_rng(42)
    plocs = np.concatenate([rng.random((120, 2)), 0.3 + 0.01 * rng.random((8, 2)), [[1.0, 1.0], [0.5, 0.25]]])
    theta = _theta(family)
    p = O.Problem(locs, y, M=len(J), J=J, r=r, family=family)
    mo, vo = O.predict(p, theta, plocs)
    with mra.Handle(locs, y, M=len(J), r=r, J=J, family=family, precision=precision) as h:
        mg, vg = h.predict(theta, plocs)
        mj, cj = h.predict_joint(theta, plocs[:60])
    tol = 1e-9 if precision == "fp64" else 1e-8
    np.testing.assert_allclose(mg, mo, rtol=tol, atol=tol * np.abs(mo).max())
    np.testing.assert_allclose(vg, vo, rtol=tol, atol=tol * np.abs(vo).max())
    mjo, cjo = O.predict_joint(p, theta, plocs[:60])
    np.testing.assert_allclose(cj, cjo, rtol=tol, atol=tol * np.abs(cjo).max())
    np.testing.assert_allclose(mj, mjo, rtol=tol, atol=tol * np.abs(mjo).max())


def test_streamed_equals_whole(mra):
    """A streamed level-1 handle (J_1 = 8 subtrees) gives the whole tree's loglik,
    gradient and kriging."""
    J, r = (8, 4, 2), 16
    locs, y = _data(3000, 51)
    plocs = np.random.default_rng(52).random((200, 2))
    theta = np.array(TH_EXP)
    with mra.Handle(locs, y, M=3, r=r, J=J, precision="emu") as hw, \
            mra.Handle(locs, y, M=3, r=r, J=J, precision="emu", stream_level=1) as hs:
        assert hs.loglik(theta) == pytest.approx(hw.loglik(theta), rel=1e-12)
        lw, gw = hw.loglik_grad(theta)
        ls, gs = hs.loglik_grad(theta)
        assert ls == pytest.approx(lw, rel=1e-12)
        np.testing.assert_allclose(gs, gw, rtol=1e-10)
        mw, vw = hw.predict(theta, plocs)
        ms, vs = hs.predict(theta, plocs)
        np.testing.assert_allclose(ms, mw, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(vs, vw, rtol=1e-10, atol=1e-12)


def test_batch_of_mixed_partitions(mra):
    rng = np.random.default_rng(61)
    datasets = []
    for k, J in enumerate([(8, 2), 4, (16, 2), (2, 2, 4)]):
        M = len(J) if not isinstance(J, int) else 2
        n = 600 + 150 * k
        locs = rng.random((n, 2))
        datasets.append({"locs": locs, "y": rng.standard_normal(n), "M": M, "J": J, "family": "exp",
                         "theta": (1.0, 0.1 + 0.05 * k, 0.05)})
    for precision in ("fp64", "emu"):
        with mra.Batch(datasets, r=16, precision=precision) as b:
            lls = b.loglik([d["theta"] for d in datasets])
        ref = [O.loglik(O.Problem(d["locs"], d["y"], M=d["M"], J=d["J"], r=16, family="exp"), d["theta"])
               for d in datasets]
        np.testing.assert_allclose(lls, ref, rtol=1e-10)


def test_two_phase_subtrees(mra):
    """The sharded two-phase evaluation (Sec. 3.5) on a level-varying tree: every
    level-1 region has J_2 = 8 children, whose (d, u) the summaries carry."""
    from paper_1507_04789_gb300 import shard
    J = (2, 8, 2)
    locs, y = _data(2000, 71)
    theta = TH_EXP
    ll_o = O.loglik(O.Problem(locs, y, M=3, J=J, r=16, family="exp"), theta)
    with mra.Handle(locs, y, M=3, r=16, J=J, precision="emu", stream_level=1) as h0, \
            mra.Handle(locs, y, M=3, r=16, J=J, precision="emu", stream_level=1) as h1:
        length, nsub = h0.summary_len()
        assert nsub == 2 and length == 3 * 16 * 16 + 2 * 16 + 2 * 8
        parts = [hk.loglik_subtrees(theta, *shard.subtree_range(nsub, k, 2)) for k, hk in enumerate((h0, h1))]
        joined = np.concatenate(parts)
        for hk in (h0, h1):
            assert hk.loglik_combine(theta, joined) == pytest.approx(ll_o, rel=1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_sequence_with_sixteen_leaves_per_parent(mra, precision):
    """Sec. 4.3's own (J_1, ..., J_6) = (2, 2, 4, 8, 8, 16): 16384 leaves, sixteen
    per level-5 region (J_M > 4 is open to the FP64 and 3xTF32 forms)."""
    J = (2, 2, 4, 8, 8, 16)
    locs, y = _data(30000, 81)
    p = O.Problem(locs, y, M=6, J=J, r=4, family="exp")
    ll_o, _, Q = O.loglik(p, TH_EXP, return_state=True)
    with mra.Handle(locs, y, M=6, r=4, J=J, family="exp", precision=precision) as h:
        off, perm = h.leaf_offsets(with_perm=True)
        assert off.shape[0] == 16385
        for i in range(0, 16384, 97):
            np.testing.assert_array_equal(perm[off[i]:off[i + 1]], p.tree.obs[i])
        ll = h.loglik(TH_EXP)
        if precision == "mixed":
            # measured 3.2e-6 per observation: r = 4 and about two observations per leaf, where the
            # 3xTF32 products' rounding weighs more per observation than on the n = 2^20, r = 64 workload
            assert abs(ll - ll_o) <= 5e-6 * 30000
            return
        assert ll == pytest.approx(ll_o, rel=1e-10)
        scale = abs(Q.d[(0, 0)]) + abs(Q.u[(0, 0)]) + 1.0
        for m in (0, 3, 5, 6):
            d_g, u_g = h.region_terms(m)
            d_o = np.array([Q.d.get((m, i), 0.0) for i in range(p.tree.nreg(m))])
            u_o = np.array([Q.u.get((m, i), 0.0) for i in range(p.tree.nreg(m))])
            np.testing.assert_allclose(d_g, d_o, rtol=1e-10, atol=1e-11 * scale)
            np.testing.assert_allclose(u_g, u_o, rtol=1e-10, atol=1e-11 * scale)


def test_sixteen_leaves_per_parent_gradient_and_prediction(mra):
    J = (2, 4, 16)
    locs, y = _data(3000, 91)
    theta = np.array(TH_M15)
    p = O.Problem(locs, y, M=3, J=J, r=9, family="matern15")
    ll_o, g_o = O.loglik_grad(p, theta)
    plocs = np.random.default_rng(92).random((150, 2))
    mo, vo = O.predict(p, tuple(theta), plocs)
    with mra.Handle(locs, y, M=3, r=9, J=J, family="matern15") as h:
        ll, g = h.loglik_grad(theta)
        mg, vg = h.predict(tuple(theta), plocs)
    assert ll == pytest.approx(ll_o, rel=1e-10)
    np.testing.assert_allclose(g, g_o, rtol=1e-8, atol=1e-8 * np.abs(g_o).max())
    np.testing.assert_allclose(mg, mo, rtol=1e-9, atol=1e-9 * np.abs(mo).max())
    np.testing.assert_allclose(vg, vo, rtol=1e-9, atol=1e-9 * np.abs(vo).max())
    with pytest.raises(mra.MRAError):
        mra.Handle(locs, y, M=3, r=9, J=J, precision="emu")

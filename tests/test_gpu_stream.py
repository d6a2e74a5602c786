"""Subtree streaming: a tree evaluated as its level-s subtrees one after another
(chunk buffers for the levels below s) gives the same log-likelihood and region
terms as the whole-tree evaluation, in the FP64 and the emulated forms, on
complete and pruned trees; and the oracle agrees with both.
"""
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


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_streamed_equals_whole_tree(mra, precision):
    w = synth.workload("n16k_matern15_M4_r64")
    locs, y, _ = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=-1) as h:
        ll = h.loglik(theta)
        terms = [h.region_terms(m) for m in range(w.M + 1)]
    for s in (1, 2, 3):
        with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=s) as hs:
            lls = hs.loglik(theta)
            assert lls == pytest.approx(ll, rel=1e-13), s
            for m in range(w.M + 1):
                d, u = hs.region_terms(m)
                np.testing.assert_allclose(d, terms[m][0], rtol=1e-12, atol=1e-12)
                np.testing.assert_allclose(u, terms[m][1], rtol=1e-12, atol=1e-12)
            assert hs.loglik((theta[0], theta[1] * 1.1, theta[2])) != lls   # a new theta is evaluated


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_streamed_gradient_equals_whole_tree(mra, precision):
    """The streamed reverse pass (coarse posterior adjoint, then per chunk its
    factors formed again and its levels' adjoints, then the coarse prior
    adjoint) gives the whole-tree gradient, at every stream level."""
    w = synth.workload("n16k_matern15_M4_r64")
    locs, y, _ = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=-1) as h:
        ll, g = h.loglik_grad(theta)
    for s in (1, 2, 3):
        with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=s) as hs:
            lls, gs = hs.loglik_grad(theta)
            assert lls == pytest.approx(ll, rel=1e-13), s
            # (FP64: the same arithmetic up to summation order; emulated: the per-parent S
            # buffer of a chunk may be left out where the whole tree's is taken, and the
            # engine's products round at about 1e-14 relative)
            tol = 1e-11 if precision == "fp64" else 1e-10
            np.testing.assert_allclose(gs, g, rtol=tol, atol=tol * np.abs(g).max(), err_msg=f"s={s}")
            # a plain evaluation and a second gradient on the same handle agree
            assert hs.loglik(theta) == pytest.approx(ll, rel=1e-13)
            lls2, gs2 = hs.loglik_grad(theta)
            np.testing.assert_allclose(gs2, gs, rtol=1e-13, atol=0)


def test_streamed_gradient_pruned_swath_matches_oracle(mra):
    """Streamed gradient on a pruned swath tree against the oracle's gradient."""
    from paper_1507_04789_gb300 import plan
    data = synth.swath_batch(1, seed=31, n_min=6e3, n_max=8e3)[0]
    locs, y = data["locs"], data["y"]
    theta = (1.0, data["kappa"], data["tau2"])
    M = plan.choose_levels(locs, 64)
    g_o = O.loglik_grad(O.Problem(locs, y, M=M, r=16, family="exp"), theta)[1]
    for precision in ("fp64", "emu"):
        with mra.Handle(locs, y, M=M, r=16, family="exp", precision=precision, prune=True, stream_level=2) as h:
            g = h.loglik_grad(theta)[1]
        np.testing.assert_allclose(g, g_o, rtol=1e-8, atol=1e-8 * np.abs(g_o).max(), err_msg=precision)


def test_streamed_pruned_swath_matches_oracle(mra):
    from paper_1507_04789_gb300 import plan
    data = synth.swath_batch(1, seed=31, n_min=6e3, n_max=8e3)[0]
    locs, y = data["locs"], data["y"]
    theta = (1.0, data["kappa"], data["tau2"])
    M = plan.choose_levels(locs, 64)
    assert M >= 3
    ll_o = O.loglik(O.Problem(locs, y, M=M, r=16, family="exp"), theta)
    for precision in ("fp64", "emu"):
        with mra.Handle(locs, y, M=M, r=16, family="exp", precision=precision, prune=True, stream_level=2) as h:
            assert h.loglik(theta) == pytest.approx(ll_o, rel=1e-10)


def test_streamed_handle_limits(mra):
    rng = np.random.default_rng(5)
    locs = rng.random((3000, 2))
    y = rng.standard_normal(3000)
    with pytest.raises(mra.MRAError) as ei:
        mra.Handle(locs, y, M=3, r=16, stream_level=3)
    assert ei.value.code == mra.MRA_ERR_ARG
    with mra.Handle(locs, y, M=3, r=16, stream_level=1) as h:
        h.loglik((1.0, 0.1, 0.01))
        for call in (lambda: h.predict_joint((1.0, 0.1, 0.01), locs[:10]), lambda: h.update(locs, y)):
            with pytest.raises(mra.MRAError) as ei:
                call()
            assert ei.value.code == mra.MRA_ERR_STATE


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_two_phase_subtrees_virtual_ranks(mra, precision):
    """The two-phase boundary of the sharded evaluation on one GPU: two handles
    (standing for two ranks, run one after the other) each evaluate their block
    of level-2 subtrees, the summaries are joined as the all-gather would join
    them, and both finish with the whole-tree log-likelihood."""
    from paper_1507_04789_gb300 import shard
    w = synth.workload("n16k_matern15_M4_r64")
    locs, y, _ = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=-1) as h:
        ll = h.loglik(theta)
        d1, u1 = h.region_terms(1)
    hs = [mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=2) for _ in range(2)]
    try:
        length, nsub = hs[0].summary_len()
        assert nsub == 16 and length == 6 * w.r * w.r + 3 * w.r + 8
        parts = [hk.loglik_subtrees(theta, *shard.subtree_range(nsub, k, 2)) for k, hk in enumerate(hs)]
        joined = np.concatenate(parts)
        for hk in hs:
            assert hk.loglik_combine(theta, joined) == pytest.approx(ll, rel=1e-13)
            d, u = hk.region_terms(1)
            np.testing.assert_allclose(d, d1, rtol=1e-12)
            np.testing.assert_allclose(u, u1, rtol=1e-12)
        assert shard.sharded_loglik(hs[0], theta, 0, 1) == pytest.approx(ll, rel=1e-13)
    finally:
        for hk in hs:
            hk.close()


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_streamed_prediction_equals_whole_tree(mra, precision):
    """Prediction on a streamed handle (each chunk's factors formed again before
    its points are predicted) equals the whole-tree prediction, and the oracle."""
    w = synth.workload("n16k_matern15_M4_r64")
    locs, y, plocs = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=-1) as h:
        m0, v0 = h.predict(theta, plocs)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision, stream_level=2) as hs:
        m1, v1 = hs.predict(theta, plocs)
        m2, _ = hs.predict(theta, plocs[:100])
    np.testing.assert_allclose(m1, m0, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(v1, v0, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(m2, m0[:100], rtol=1e-12, atol=1e-13)

"""FP64-emulation form (every large contraction on the bf16 tensor cores as
seven 7-bit slices per operand) against the FP64 oracle.

Each emulated product carries about 1e-14 relative error (operands truncated to
49 bits below their 64-column group's largest element, double-float sums).  The
prior chain cancels by up to 1e5 at the finest levels, which the FP64 form
shares; measured, the emulated form stays within the FP64 form's own bars: a
relative 1e-10 on the log-likelihood and 1e-9 on predictions, on uniform data
and on the dense swath data where the 3xTF32 form loses most.
"""
import numpy as np
import pytest

from oracle import mra_oracle as O
from paper_1507_04789_gb300 import plan, synth

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-10
PRED_RTOL = 1e-9


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


@pytest.mark.parametrize("name", ["n4096_exp_M3_r16", "n16k_matern15_M4_r64"])
def test_emu_loglik_matches_oracle(mra, name):
    w = synth.workload(name)
    locs, y, plocs = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    ll_o = O.loglik(p, theta)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision="emu") as h:
        ll = h.loglik(theta)
        err = abs(ll - ll_o) / abs(ll_o)
        print(f"{name}: emu loglik {ll:.12f} oracle {ll_o:.12f} rel {err:.3e}")
        assert err <= LL_RTOL
        assert h.loglik(theta) == ll                     # deterministic
        mean, var = h.predict(theta, plocs[:256])
    mo, vo = O.predict(p, theta, plocs[:256])
    em = np.abs(mean - mo).max() / np.abs(mo).max()
    ev = np.abs(var - vo).max() / np.abs(vo).max()
    print(f"{name}: prediction max rel err mean {em:.3e} var {ev:.3e}")
    assert em <= PRED_RTOL and ev <= PRED_RTOL


@pytest.mark.parametrize("name", ["n4096_exp_M3_r16", "n16k_matern15_M4_r64"])
def test_emu_gradient(mra, name):
    """Hbar = 2 H S + z omegabar' on the tensor cores: one 48-column group per
    row (M r = 48), and two 128-column groups with ragged 128-row tiles of each
    parent's rows (M r = 256)."""
    w = synth.workload(name)
    locs, y, _ = w.generate()
    theta = np.array([w.sigma2, w.kappa, w.tau2])
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    _, g_o = O.loglik_grad(p, theta)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision="emu") as h:
        _, g = h.loglik_grad(theta)
    rel = np.abs(g - g_o).max() / np.abs(g_o).max()
    print(f"{name}: emu gradient max rel err {rel:.3e}")
    assert rel <= 1e-8                                   # the FP64 form's gradient bar


def test_emu_gradient_pruned_tree_and_memory_rule(mra):
    """Clustered data, M = 4, r = 48: column blocks of S straddle the 128-column
    scale groups.  On the complete tree the per-parent S would take more than
    four times the memory of H and the leaf adjoint forms Hbar in FP64; on the
    pruned tree (20 of 64 parents) the tensor cores form it."""
    rng = np.random.default_rng(21)
    locs = np.concatenate([0.25 * rng.random((1200, 2)), 0.6 + 0.4 * rng.random((1700, 2))])
    y = synth.noisy_observations(synth.rff_field(locs, 1.5, 0.1, 1.0, 4), 0.05, 9)
    theta = np.array([1.0, 0.1, 0.05])
    ll_o, g_o = O.loglik_grad(O.Problem(locs, y, M=4, r=48, family="matern15"), theta)
    for prune in (False, True):
        with mra.Handle(locs, y, M=4, r=48, family="matern15", precision="emu", prune=prune) as h:
            ll, g = h.loglik_grad(theta)
        rel = np.abs(g - g_o).max() / np.abs(g_o).max()
        print(f"prune={prune}: emu gradient max rel err {rel:.3e}")
        assert ll == pytest.approx(ll_o, rel=LL_RTOL)
        assert rel <= 1e-8


def test_emu_region_terms_and_ragged(mra):
    """Ragged leaves (several 64-column groups and a tail), a pruned tree and
    per-region terms against the FP64 kernels."""
    rng = np.random.default_rng(21)
    locs = np.concatenate([0.25 * rng.random((1200, 2)), 0.6 + 0.4 * rng.random((1700, 2))])
    y = synth.noisy_observations(synth.rff_field(locs, 1.5, 0.1, 1.0, 4), 0.05, 9)
    theta = (1.0, 0.1, 0.05)
    for prune in (False, True):
        with mra.Handle(locs, y, M=4, r=48, family="matern15", prune=prune) as h64, \
                mra.Handle(locs, y, M=4, r=48, family="matern15", precision="emu", prune=prune) as he:
            a, b = h64.loglik(theta), he.loglik(theta)
            print(f"prune={prune}: rel d loglik = {abs(a - b) / abs(a):.3e}")
            assert b == pytest.approx(a, rel=LL_RTOL)
            for m in range(5):
                d64, u64 = h64.region_terms(m)
                de, ue = he.region_terms(m)
                np.testing.assert_allclose(de, d64, rtol=1e-8, atol=1e-9 * max(1.0, np.abs(d64).max()))
                np.testing.assert_allclose(ue, u64, rtol=1e-8, atol=1e-9 * max(1.0, np.abs(u64).max()))


def test_emu_batch_on_swath_data(mra):
    """Dense swath data, where the 3xTF32 form's error reaches 1e-6 per observation."""
    data = synth.swath_batch(4, seed=12, n_min=1.5e3, n_max=1.2e4)
    datasets = [{"locs": d["locs"], "y": d["y"], "M": plan.choose_levels(d["locs"], 64),
                 "family": "exp" if k % 2 == 0 else "matern15", "theta": (1.0, d["kappa"], d["tau2"])}
                for k, d in enumerate(data)]
    thetas = [d["theta"] for d in datasets]
    ref = np.array([O.loglik(O.Problem(d["locs"], d["y"], M=d["M"], r=32, family=d["family"]), d["theta"])
                    for d in datasets])
    with mra.Batch(datasets, r=32, precision="emu") as be:
        c = be.loglik(thetas)
        assert np.array_equal(be.loglik(thetas), c)     # graph replay is deterministic
    print("emu batch relative error:", np.abs(ref - c) / np.abs(ref))
    np.testing.assert_allclose(c, ref, rtol=LL_RTOL)


def test_emu_gradient_without_optional_buffers(mra):
    """MRA_OPT_GRAD_BUFFERS = 0: no per-parent S and no stored C0 derivatives, so
    Hbar and Gbar come from the FP64 kernels and the chain adjoint evaluates the
    covariance derivatives itself; the gradient still meets the oracle's bar and
    equals the buffered form's to rounding."""
    w = synth.workload("n16k_matern15_M4_r64")
    locs, y, _ = w.generate()
    theta = np.array([w.sigma2, w.kappa, w.tau2])
    _, g_o = O.loglik_grad(O.Problem(locs, y, M=w.M, r=w.r, family=w.family), theta)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision="emu") as h:
        ll1, g1 = h.loglik_grad(theta)
        h.set_option(mra.MRA_OPT_GRAD_BUFFERS, 0)
        ll0, g0 = h.loglik_grad(theta)
        h.set_option(mra.MRA_OPT_GRAD_BUFFERS, 1)
        ll2, g2 = h.loglik_grad(theta)
    for g in (g0, g1):
        assert np.abs(g - g_o).max() / np.abs(g_o).max() <= 1e-8
    assert ll0 == ll1 == ll2
    np.testing.assert_array_equal(g1, g2)
    np.testing.assert_allclose(g0, g1, rtol=1e-10, atol=1e-10 * np.abs(g1).max())

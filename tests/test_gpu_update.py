"""mra_update on an existing handle (new locations and data, same n): the
log-likelihood equals that of a handle built on the new data, in every form,
including the emulated form's groups of leaves and of sibling regions, which
follow the new occupancy."""
import numpy as np
import pytest

from paper_1507_04789_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_update_equals_fresh_build(mra, precision):
    rng = np.random.default_rng(11)
    n = 6000
    # sparse, clustered first data (small parents: the emulated form groups them), then uniform data
    a = synth.swath_batch(1, seed=5, n_min=n, n_max=n + 1)[0]
    locs1 = a["locs"][:n]
    y1 = a["y"][:n]
    locs2 = rng.random((len(locs1), 2))
    y2 = rng.standard_normal(len(locs1))
    from paper_1507_04789_gb300 import plan
    theta = (1.0, 0.1, 0.05)
    kw = dict(M=plan.choose_levels(locs1, 64), r=16, family="exp", precision=precision)
    with mra.Handle(locs1, y1, **kw) as h:
        h.loglik(theta)
        h.update(locs2, y2)
        ll_upd = h.loglik(theta)
        h.update(locs1, y1)
        ll_back = h.loglik(theta)
    with mra.Handle(locs2, y2, **kw) as h2:
        ll_new = h2.loglik(theta)
    with mra.Handle(locs1, y1, **kw) as h1:
        ll_old = h1.loglik(theta)
    assert ll_upd == pytest.approx(ll_new, rel=1e-14, abs=0)
    assert ll_back == pytest.approx(ll_old, rel=1e-14, abs=0)

"""mra_stats: per-level time and algorithmic work of an evaluation.

The library's FLOP model (per level and stage) is checked against the one
bench.py states for the roofline (written separately), per stage; the timed
launches must be one per level and stage per evaluation, with positive times.
"""
import numpy as np
import pytest

import bench
from paper_1507_04789_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mra():
    from paper_1507_04789_gb300 import mra as m
    m.load_library()
    return m


@pytest.mark.parametrize("precision", ["fp64", "emu"])
def test_stats_flops_and_times(mra, precision):
    w = synth.workload("n16k_matern15_M4_r64")
    locs, y, _ = w.generate()
    theta = (w.sigma2, w.kappa, w.tau2)
    with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision) as h:
        h.enable_timing(True)
        for _ in range(2):
            h.loglik(theta)
        st = h.stats()
        off = h.leaf_offsets()
    nF = np.diff(off)
    ref = bench.algorithmic_flops(w.M, w.r, nF)
    M = w.M
    assert st["M"] == M and st["evaluations"] == 2
    lv = st["levels"]
    tot = {k: 0.0 for k in ref}
    for m in range(M + 1):
        for name, v in lv[m].items():
            key = "leaf" if name == "chain" else name
            tot[key] += v["flops"]
            assert v["launches"] == 2 and v["ms"] > 0.0, (m, name, v)
            assert v["bytes"] > 0.0 and v["units"] > 0.0
    for k in ref:
        assert tot[k] == pytest.approx(ref[k], rel=1e-12), k
    for m in range(M):
        assert lv[m]["prior"]["units"] == 4 ** m and lv[m]["post"]["units"] == 4 ** m
    assert ("chain" in lv[M]) == (precision == "emu")
    assert lv[M]["leaf"]["units"] == 4 ** M

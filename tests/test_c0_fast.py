"""The covariance kernels' C0 with few FP64 operations (mra_device.cuh
c0_fast: a double-float square-root seed and one FP64 Newton step, a
4096-entry table exponential with a double-float polynomial), compiled for the
host, against 40-digit values of sigma2 e^{-a} and sigma2 (1 + a) e^{-a},
a = sqrt(u): within 4 ulp plus a/2 ulp (the rounding of a itself), over
distances from 2^-29 to the cut at a = 708, variance factors from 1e-3 to 1e3,
and the special cases (u = 0, tiny u, a beyond 708)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def c0_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("c0") / "c0_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-o", exe,
                    os.path.join(HERE, "c0_check.cu")], check=True, capture_output=True)
    return exe


def _run(exe, rows):
    inp = "\n".join(f"{f} {float(u).hex()} {float(s).hex()}" for f, u, s in rows)
    out = subprocess.run([exe], input=inp, check=True, capture_output=True, text=True).stdout
    return np.array([float.fromhex(v) for v in out.split()])


def _ref(mp, family, u, sc):
    a = mp.sqrt(mp.mpf(u))
    e = mp.exp(-a)
    return mp.mpf(sc) * (e if family == 0 else (1 + a) * e)


def test_c0_fast_against_high_precision(c0_exe):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(3)
    a = np.concatenate([10.0 ** rng.uniform(-9, np.log10(700.0), 3000),
                        rng.uniform(0.0, 3.0, 1000),               # the range that dominates the blocks
                        np.arange(1, 200) * float(mp.log(2) / 4096)])   # reduction boundaries
    rows = []
    for i, ai in enumerate(a):
        rows.append((i % 2, float(ai) ** 2, float(10.0 ** rng.uniform(-3, 3))))
    got = _run(c0_exe, rows)
    worst = 0.0
    for (f, u, sc), g in zip(rows, got):
        ref = _ref(mp, f, u, sc)
        if ref == 0:
            assert g == 0.0
            continue
        err = float(abs(mp.mpf(g) - ref) / ref) / 2.0 ** -53
        ai = float(mp.sqrt(u))
        worst = max(worst, err / (4.0 + 0.5 * ai))
        assert err <= 4.0 + 0.5 * ai, (f, u, sc, g, float(ref), err)
    assert worst > 0.0


def test_c0_fast_special_cases(c0_exe):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rows = [(0, 0.0, 2.0), (1, 0.0, 2.0), (0, 2.0 ** -80, 1.5), (1, 2.0 ** -80, 1.5), (0, 2.0 ** -62, 1.0),
            (1, 2.0 ** -62, 1.0), (0, 709.0 ** 2, 1.0), (1, 1e12, 1.0), (0, 700.0 ** 2, 1.0)]
    got = _run(c0_exe, rows)
    assert got[0] == 2.0 and got[1] == 2.0
    for (f, u, sc), g in list(zip(rows, got))[2:6]:
        ref = _ref(mp, f, u, sc)
        assert abs(g - float(ref)) <= 4 * 2.0 ** -53 * float(ref)
    assert got[6] == 0.0 and got[7] == 0.0
    assert got[8] == pytest.approx(float(_ref(mp, 0, 700.0 ** 2, 1.0)), rel=1e-12)

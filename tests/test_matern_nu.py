"""The free-smoothness Matern correlation the kernels evaluate (trapezoidal
rule for K_nu, mra_device.cuh matern_nu), compiled for the host, against the
library Bessel function (scipy.special.kv) and its closed forms at half-integer
smoothness: rho within 1e-12 relative, d rho / d h and d rho / d nu within
1e-11 of their 40-digit values (mpmath)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.special import gamma, kv

HERE = os.path.dirname(os.path.abspath(__file__))


def ref_rho(nu, h):
    z = math.sqrt(2.0 * nu) * h
    return 2.0 ** (1.0 - nu) / gamma(nu) * z ** nu * kv(nu, z)


@pytest.fixture(scope="module")
def matern_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("mat") / "matern_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-o", exe,
                    os.path.join(HERE, "matern_check.cu")], check=True, capture_output=True)
    return exe


def _run(exe, pairs):
    inp = "\n".join(f"{float(nu):.17g} {float(h):.17g}" for nu, h in pairs)
    out = subprocess.run([exe], input=inp, check=True, capture_output=True, text=True).stdout
    return np.array([[float(v) for v in ln.split()] for ln in out.strip().splitlines()])


def test_matern_nu_values_and_derivatives(matern_exe):
    """Values against scipy's kv; derivatives against 40-digit mpmath:
    d rho / dh = -c_nu sqrt(2 nu) z^nu K_{nu-1}(z) and d rho / d nu by mpmath.diff."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    pairs = [(nu, h) for nu in (0.3, 0.5, 0.8, 1.5, 2.2, 2.5, 3.7, 6.0)
             for h in (1e-7, 1e-4, 1e-2, 0.05, 0.2, 0.7, 1.5, 4.0, 12.0, 40.0)]
    got = _run(matern_exe, pairs)

    def rho_mp(nu, h):
        z = mp.sqrt(2 * nu) * h
        return 2 ** (1 - nu) / mp.gamma(nu) * z ** nu * mp.besselk(nu, z)

    worst = 0.0
    for (nu, h), (rho, dh, dnu) in zip(pairs, got):
        ref = ref_rho(nu, h)
        assert rho == pytest.approx(ref, rel=1e-12, abs=1e-300), (nu, h)
        n_, h_ = mp.mpf(nu), mp.mpf(h)
        z = mp.sqrt(2 * n_) * h_
        rdh = float(-2 ** (1 - n_) / mp.gamma(n_) * mp.sqrt(2 * n_) * z ** n_ * mp.besselk(n_ - 1, z))
        rdn = float(mp.diff(lambda v: rho_mp(v, h_), n_))
        assert dh == pytest.approx(rdh, rel=1e-11, abs=1e-300), (nu, h, dh, rdh)
        assert abs(dnu - rdn) <= 1e-11 * max(abs(rdn), abs(ref)), (nu, h, dnu, rdn)
        worst = max(worst, abs(rho - ref) / ref)
    print("worst relative error of rho:", worst)


def test_matern_nu_half_integers_and_origin(matern_exe):
    h = np.array([1e-3, 0.1, 0.5, 1.0, 2.0, 5.0])
    got = _run(matern_exe, [(0.5, v) for v in h] + [(1.5, v) for v in h] + [(2.5, v) for v in h] + [(1.7, 0.0)])
    s3, s5 = math.sqrt(3.0), math.sqrt(5.0)
    np.testing.assert_allclose(got[:6, 0], np.exp(-h), rtol=1e-12)
    np.testing.assert_allclose(got[6:12, 0], (1 + s3 * h) * np.exp(-s3 * h), rtol=1e-12)
    np.testing.assert_allclose(got[12:18, 0], (1 + s5 * h + 5 * h * h / 3) * np.exp(-s5 * h), rtol=1e-12)
    np.testing.assert_array_equal(got[18], [1.0, 0.0, 0.0])

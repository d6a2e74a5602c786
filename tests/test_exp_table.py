"""The covariance exponential e^{-a} (table-driven argument reduction, Tang
1989; degree-5 Taylor polynomial) against long double expl, on the host:
the same source the kernels compile, checked to 2.5 ulp (2^-53 = 1.1e-16)."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_exp_neg_within_ulps(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "exp_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-o", exe,
                    os.path.join(HERE, "exp_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    m = re.search(r"max_rel ([0-9.e+-]+) .* edges_ok (\d)", out)
    assert m, out
    assert float(m.group(1)) <= 2.5 * 2.0 ** -53, out
    assert m.group(2) == "1", out

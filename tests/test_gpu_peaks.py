"""Peak rates of the pipes the kernels run on (FP64 FMA, FP64 mma.sync, and
the engines' own tcgen05 MMA shapes), timed with CUDA events with the SM clock
sampled meanwhile; the roofline denominators for the FP64 kernels and the
ceiling of the engines' MMA shapes against the measured cuBLAS bf16 peak."""
import json
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_pipe_peaks(tmp_path):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "peaks")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "paper_1507_04789_gb300", "csrc"),
                    "-o", exe, os.path.join(HERE, "peaks.cu")], check=True, capture_output=True)
    clk = bench.ClockSampler(0)
    clk.start()
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    clocks = clk.stop()
    assert res.returncode == 0, res.stdout + res.stderr
    d = json.loads(res.stdout.strip().splitlines()[-1])
    d["clocks"] = clocks
    print(json.dumps(d))
    assert 0.3 < d["dfma_tflops"] < 3.0
    assert 0.1 < d["dmma_tflops"] < 5.0
    assert 100.0 < d["bf16_128x64x16_tflops"] < 3000.0
    assert 50.0 < d["tf32_128x64x8_tflops"] < 2000.0

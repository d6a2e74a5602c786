"""Host-side logic of bench.py, on the CPU: the reference arm's JSON line
(single process and two ranks under torchrun, where rank 0 alone reports), the
traffic guard that drops a DRAM figure once the kernel sources change, and the
FLOP models the roofline divides by."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--workload", "n4096_exp_M3_r16", "--steps", "1", "--warmup", "3"]


def _json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def _check_reference_line(d, n_gpus):
    assert d["impl"] == "reference"
    assert d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(1e3 / d["value"])
    assert d["n_gpus"] == n_gpus and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"] == "n4096_exp_M3_r16"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_line():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", *SMALL], cwd=ROOT,
                         capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = _json_lines(res.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_two_ranks():
    with socket.socket() as s:   # a free port for the rendezvous
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", *SMALL]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = _json_lines(res.stdout)
    assert len(lines) == 1                       # rank 0 alone reports; rank 1 exits without work
    _check_reference_line(lines[0], 2)


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_traffic_guard(monkeypatch):
    bench = _bench()
    assert bench.kernel_traffic("emu", "no-such-kernel", "n1M_matern15_M7_r64") == (None, None)
    fake = {("emu", "leaf", "w"): {"bytes": 1.0, "how": "x", "sources": ["mra_emu.cuh"], "sha1": "0" * 40}}
    monkeypatch.setattr(bench, "TRAFFIC", fake)
    b, how = bench.kernel_traffic("emu", "leaf", "w")
    assert b is None and "changed" in how


def test_flop_models():
    bench = _bench()
    rng = np.random.default_rng(3)
    for M, r in ((1, 8), (3, 16), (4, 32)):
        nF = rng.integers(20, 90, size=4 ** M)
        alg = bench.algorithmic_flops(M, r, nF)
        for prec in ("emu", "mixed"):
            cf = bench.contraction_flops(M, r, nF, prec)
            for k, v in cf.items():
                assert 0 <= v <= alg[k] * (1 + 1e-12), (M, r, prec, k)
        # the Gram product of the leaves is linear in the observations under each parent
        alg2 = bench.algorithmic_flops(M, r, 2 * nF)
        assert alg2["leaf_syrk"] == pytest.approx(2 * alg["leaf_syrk"])


def test_per_level_models():
    """The contraction part of every (level, stage) stays within its algorithmic
    FLOPs as the library's model counts them (here the bench's own per-kind
    model, split by level), and the prediction model grows with the leaf size."""
    bench = _bench()
    rng = np.random.default_rng(4)
    for M, r in ((2, 16), (4, 64)):
        nF = rng.integers(20, 90, size=4 ** M)
        alg = bench.algorithmic_flops(M, r, nF)
        tot = {k: 0.0 for k in alg}
        for m in range(M):
            tot["prior"] += bench.contraction_share("prior", m, M, r, nF)
            tot["post"] += bench.contraction_share("post", m, M, r, nF)
            if m > 0:
                tot["aggregate"] += bench.contraction_share("aggregate", m, M, r, nF)
        tot["leaf"] = bench.contraction_share("chain", M, M, r, nF) + bench.contraction_share("leaf", M, M, r, nF)
        tot["leaf_syrk"] = bench.contraction_share("leaf_syrk", M, M, r, nF)
        for k in alg:
            assert 0 < tot[k] <= alg[k], (M, r, k)
    assert bench.predict_flops_per_point(7, 64, 80.0) > bench.predict_flops_per_point(7, 64, 40.0) > 0

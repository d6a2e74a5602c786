#!/usr/bin/env python
"""Benchmark of the M-RA log-likelihood on GB300 (prints one JSON line).

One step = one log-likelihood evaluation of the whole hot path at a new
parameter value: the prior pass over every level, the leaf factorisation, the
leaf Gram products, the posterior pass and the root scalar (Sec. 3.1-3.3).
The workload is n = 2^20 uniform locations on [0,1]^2 with a Matern-1.5 field
(sigma2 = 1, range 0.1, tau2 = 0.01), M = 7, J = 4, r = 64 (about 64
observations per leaf).  Three forms are timed on the same steps:

  fp64   every product on the FP64 pipe
  mixed  prior and leaf contractions on the tensor cores as 3xTF32
  emu    every large contraction (prior, leaf and both Gram products) on the
         tensor cores as a bf16-slice FP64 emulation (about 1e-14 per product)

The headline is the fastest form whose log-likelihoods stay within
|d loglik| / n <= 1e-6 of the FP64 form; the others are reported beside it,
together with loglik + gradient evaluations ("gradient": the emulated form, forward and adjoint on the
FP64 emulation, beside the FP64 form). `--grad-only` times only the emulated loglik + gradient.

  value        evals/s with the inputs resident in HBM (CUDA events on the
               library's stream, max over ranks)
  e2e          the same metric through the C ABI with host inputs: every step
               copies locations and data from pinned host memory, re-partitions
               them on the device and reads the result back
  roofline     the dominant kernel of the headline form: for a tensor-core
               kernel, the bf16 (emu) or TF32 (mixed) tensor FLOP/s its
               contractions need (algorithmic FP64 MACs x slice products) over
               its CUDA-event time, against the measured bf16 peak (TF32 at the
               nominal TF32/bf16 ratio); for an FP64 kernel, algorithmic FP64
               FLOP/s against the FP64 pipe's peak
  cpu_baseline the FP64 CPU oracle (numpy, one thread) on one level-2 subtree
               of the same problem (1/16 of the leaves), scaled to evals/s

``--impl reference`` times the oracle alone on the same workload (a bounded
sample per step) and prints the same line with "impl": "reference".

Launched with torchrun for N > 1, the ranks evaluate ONE problem together
(paper_1507_04789_gb300.shard, Sec. 3.5): every rank builds the same streamed
handle (stream_level 2: 16 level-2 subtrees), evaluates its contiguous share
of the subtrees, the ranks all-gather the subtrees' summaries over NCCL (about
3 MB, the only collective) and every rank finishes the coarse levels; value =
evaluations of the whole problem per second (strong scaling: the total work
is fixed).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "M-RA loglik(+grad) evals/s at n=2^20, mixed vs FP64 plain; % of TC/FP64 peak"
WORKLOAD = "n1M_matern15_M7_r64"
FP64_PEAK_TFLOPS = 1.10     # GB300 FP64 pipe, measured: DMMA m8n8k4 1.103, DFMA 1.059 TFLOP/s (tests/peaks.cu)
BF16_PEAK_FALLBACK = 1900.0  # TFLOP/s, used only without a measured peak file
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 / bf16 tensor rates
EMU_PAIRS = 28               # bf16 slice products per emulated FP64 MAC (7 slices, weights t <= 8)
TF32_PAIRS = 3               # TF32 products per 3xTF32 MAC
ORACLE_SAMPLE_LEVEL = 3     # cpu baseline: level-3 subtrees, 1/64 of the leaves each


# ---------------------------------------------------------------------------
# algorithmic FP64 work per kernel kind (MAC = 2 flops; symmetric and
# triangular products counted once)
# ---------------------------------------------------------------------------

def algorithmic_flops(M: int, r: int, nF):
    """FLOPs per log-likelihood evaluation by kernel kind."""
    import numpy as np
    nF = np.asarray(nF, dtype=np.float64)
    tri = r * (r + 1) / 2.0
    out = {"prior": 0.0, "leaf": 0.0, "leaf_syrk": 0.0, "post": 0.0, "aggregate": 0.0}
    for m in range(M):
        R = 4.0 ** m
        per = 0.0
        for l in range(m):
            per += 2.0 * r * r * (l * r) + 2.0 * r * tri      # X update, X L_l^{-T}
        per += 2.0 * tri * (m * r)                           # W = C - V V'
        per += 2.0 * r ** 3 / 3.0                            # Cholesky + triangular inverse
        out["prior"] += R * per
    Mr = M * r
    c = nF
    leaf = np.zeros_like(c)
    for l in range(M):
        leaf += 2.0 * c * r * (l * r) + 2.0 * c * tri
    leaf += c * (c + 1) * Mr                                 # Sigma = C - V V'
    leaf += 2.0 * c ** 3 / 3.0                               # Cholesky + inverse
    leaf += c * (c + 1)                                      # z
    leaf += M * r * c * (c + 1)                              # H = L^{-1} V (triangular)
    out["leaf"] = float(leaf.sum())
    if M > 0:
        rows = c.reshape(-1, 4).sum(axis=1)                  # observations per level-(M-1) parent
        out["leaf_syrk"] = float(((Mr * (Mr + 1)) * rows + 2.0 * Mr * rows).sum())
    for m in range(M):
        R = 4.0 ** m
        out["post"] += R * (2.0 * r ** 3 / 3.0 + m * r * r * (r + 1) + r * (r + 1))
        if m > 0:
            P = 4.0 ** (m - 1)
            mr = m * r
            out["aggregate"] += P * (mr * (mr + 1) * 4 * r + 2.0 * mr * 4 * r)
    return out


def contraction_flops(M: int, r: int, nF, precision: str):
    """The part of algorithmic_flops that a tensor-core form runs on the tensor
    cores (everything but the factorisations, inverses and vector terms)."""
    import numpy as np
    if precision == "fp64":
        return {}
    full = algorithmic_flops(M, r, nF)
    c = np.asarray(nF, dtype=np.float64)
    out = {"prior": full["prior"] - sum(4.0 ** m * 2.0 * r ** 3 / 3.0 for m in range(M)),
           "leaf": full["leaf"] - float((2.0 * c ** 3 / 3.0 + c * (c + 1)).sum())}
    if precision == "emu":
        Mr = M * r
        rows = c.reshape(-1, 4).sum(axis=1) if M > 0 else c
        out["leaf_syrk"] = float((Mr * (Mr + 1) * rows).sum()) if M > 0 else 0.0
        out["aggregate"] = sum(4.0 ** (m - 1) * (m * r) * (m * r + 1) * 4 * r for m in range(1, M))
    return out


# DRAM bytes per launch (per stage, where the dominant entry is a stage of two
# kernels) of the dominant kernel, from one ncu capture, valid only
# while the kernel's sources are the ones it was taken from (else null).
SOURCES_EMU = ["mra_mixed.cu", "mra_emu.cuh", "mra_tc.cuh", "mra_device.cuh", "mra_kernels.cuh"]
TRAFFIC = {
    ("emu", "chain_forward_kernel_em", "n1M_matern15_M7_r64"): {
        "bytes": 5.8848e+09,
        "how": "dram__bytes_read.sum + dram__bytes_write.sum of chain_forward_kernel_em (496.9 + 764.1 MB) "
               "at n = 2^18, M = 6 (profiles/leaf_stage_emu_n256k_matern15_M6_r64.md), scaled by n M r "
               "(x 4.667) to n = 2^20, M = 7; the kernel writes V_F (8 B x n x M r) and reads the points "
               "and the ancestors' factors, both in proportion to n M r",
        "sources": SOURCES_EMU,
        "sha1": "b81bedf3ad29b200868afd73e315bd8a28f3e961",
    },
    ("emu", "leaf_kernel_tc<1>", "n1M_matern15_M7_r64"): {
        "bytes": 8.0241e+09,
        "how": "dram__bytes_read.sum + dram__bytes_write.sum of leaf_kernel_tc<1> (824.8 + 894.6 MB) at "
               "n = 2^18, M = 6 (profiles/leaf_stage_emu_n256k_matern15_M6_r64.md), scaled by n M r (x 4.667) "
               "to n = 2^20, M = 7; the kernel reads V_F and writes H (8 B x n x M r each) and the "
               "L_Sigma^{-1} blocks (8 B x sum n_F^2, about 1/7 of it)",
        "sources": SOURCES_EMU,
        "sha1": "b81bedf3ad29b200868afd73e315bd8a28f3e961",
    },
}


def kernel_traffic(form: str, kernel: str, workload: str):
    import hashlib
    t = TRAFFIC.get((form, kernel, workload))
    if t is None:
        return None, None
    h = hashlib.sha1()
    for f in t["sources"]:
        with open(os.path.join(ROOT, "paper_1507_04789_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != t["sha1"]:
        return None, "kernel sources changed since the ncu capture"
    return t["bytes"], t["how"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle sample: level-k subtrees of the same problem on every host core
# (a spawn pool of one-BLAS-thread processes, started before any GPU work)
# ---------------------------------------------------------------------------

_POOL_PROB = None


def _pool_init(workload: str, seed: int) -> None:
    global _POOL_PROB
    from oracle import mra_oracle as O
    from paper_1507_04789_gb300 import synth
    w = synth.workload(workload)
    w = synth.Workload(**{**w.__dict__, "seed": seed})
    locs, y, _ = w.generate()
    p = O.Problem(locs, y, M=w.M, r=w.r, family=w.family)
    _ = p.tree
    _POOL_PROB = (p, (w.sigma2, w.kappa, w.tau2))


def _pool_subtree(task):
    from oracle import mra_oracle as O
    level, k = task
    p, theta = _POOL_PROB
    t0 = time.perf_counter()
    d, u = O.region_terms(p, theta, level, k)
    return k, float(d), float(u), time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


class OraclePool:
    """The oracle on `workers` host processes, each holding the problem once."""

    def __init__(self, workload: str, seed: int, workers: int):
        import multiprocessing as mp
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "CUDA_VISIBLE_DEVICES")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                           "CUDA_VISIBLE_DEVICES": ""})
        try:
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_pool_init, initargs=(workload, seed))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.workers = workers
        self.pool.map(time.sleep, [0.0] * workers)     # every worker has built its problem

    def subtrees(self, level: int, ks):
        t0 = time.perf_counter()
        res = self.pool.map(_pool_subtree, [(level, k) for k in ks], chunksize=1)
        return res, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def pool_workers(level: int) -> int:
    """One process per core, at most one per subtree and, at about 0.5 GB of
    oracle state per level-3 subtree at n = 2^20, within half the host memory."""
    try:
        mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES") / 2 ** 30
    except (ValueError, OSError, AttributeError):
        mem_gb = 16.0
    return max(1, min(host_cores(), 4 ** level, int(mem_gb / 2 / 1.0)))


def oracle_sample(workload: str, level: int, seed: int):
    """cpu_baseline: `workers` level-`level` subtrees (one per process) timed
    together; evals/s = (subtrees / 4^level) / wall time.  Also returns the
    sampled regions' d_R, u_R for the oracle error of the GPU forms."""
    workers = pool_workers(level)
    pool = OraclePool(workload, seed, workers)
    try:
        res, wall = pool.subtrees(level, range(workers))
    finally:
        pool.close()
    frac = workers / 4 ** level
    cpu_s = sum(r[3] for r in res)
    out = {"value": frac / wall, "unit": "evals/s", "cores": workers, "kind": "oracle",
           "cpu_model": host_cpu_model(), "host_cores": host_cores(),
           "sample": f"prior+posterior of {workers} level-{level} subtrees ({workers}/{4 ** level} of the leaves, "
                     f"one per process on {workers} cores, {wall:.2f} s wall, {cpu_s:.1f} s CPU) scaled to one "
                     f"evaluation; numpy FP64, one BLAS thread per process"}
    terms = {"level": level, "regions": [r[0] for r in res], "d": [r[1] for r in res], "u": [r[2] for r in res]}
    return out, terms


# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1507_04789_gb300 import synth
    level = min(ORACLE_SAMPLE_LEVEL, synth.workload(args.workload).M)
    workers = pool_workers(level)
    t_all = time.perf_counter()
    pool = OraclePool(args.workload, 0, workers)
    per = []
    try:
        for k in range(args.warmup + args.steps):
            ks = [(k * workers + j) % 4 ** level for j in range(workers)]
            _, wall = pool.subtrees(level, ks)
            if k >= args.warmup:
                per.append((workers / 4 ** level) / wall)
    finally:
        pool.close()
    value = statistics.median(per)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": workers, "kind": "oracle",
                         "cpu_model": host_cpu_model(), "host_cores": host_cores(),
                         "sample": f"per step {workers} level-{level} subtrees ({workers}/{4 ** level} of the "
                                   f"leaves, one per process on {workers} cores) scaled to one evaluation; "
                                   f"numpy FP64, one BLAS thread per process"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, world, rank, mra, np, torch):
    """64 independent swath datasets (n log-uniform in [1e4, 1e6], r = 32,
    exponential covariance with per-dataset range), pruned trees, one launch
    per level, replayed as a CUDA graph; FP64 and FP64-emulation forms."""
    from paper_1507_04789_gb300 import plan, synth
    data = synth.swath_batch(args.batch_datasets, seed=7 + rank, features=64)
    datasets = [{"locs": d["locs"], "y": d["y"], "M": plan.choose_levels(d["locs"], 64), "family": "exp"}
                for d in data]
    thetas = [(d["sigma2"], d["kappa"], d["tau2"]) for d in data]
    ns = [len(d["y"]) for d in datasets]
    out = {"workload": f"{len(datasets)} swath datasets, n log-uniform in [1e4, 1e6], r = 32, exponential, "
                       f"pruned trees", "datasets": len(datasets), "total_n": int(sum(ns)),
           "M_range": [min(d["M"] for d in datasets), max(d["M"] for d in datasets)],
           "timing": "host wall clock around graph replays (each ends in a stream sync)"}
    lls = {}
    for prec in ("fp64", "emu"):
        b = mra.Batch(datasets, r=32, precision=prec)
        t0 = time.perf_counter()
        b.loglik(thetas)                      # autotune + graph capture
        t_first = time.perf_counter() - t0
        reps = 3
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(reps):
            lls[prec] = b.loglik([(t[0], t[1] * (1.0 + 0.01 * k), t[2]) for t in thetas])
        dt = (time.perf_counter() - t0) / reps
        nd, tile = b.info()
        # one more evaluation with per-launch events (direct launches, not the graph): time per stage
        b.enable_timing(True)
        b.loglik(thetas)
        st = b.stats()
        b.enable_timing(False)
        b.close()
        stages = {}
        for row in st["levels"]:
            for k, v in row.items():
                stages[k] = stages.get(k, 0.0) + v["ms"] / max(1, st["evaluations"])
        out[prec] = {"ms_per_batch": dt * 1e3, "dataset_evals_per_s": world * nd / dt, "autotuned_tile": tile,
                     "first_call_s": t_first, "stage_ms": {k: round(v, 2) for k, v in stages.items()}}
    out["emu_max_rel_dloglik_vs_fp64"] = float(np.max(np.abs(lls["emu"] - lls["fp64"]) / np.abs(lls["fp64"])))
    return out


# Stages whose contractions run on the tensor cores in each form (the others on the FP64 pipe).
TENSOR_STAGES = {"fp64": set(), "mixed": {"prior", "leaf"},
                 "emu": {"prior", "chain", "leaf", "leaf_syrk", "post", "aggregate"}}
STAGE_KERNEL = {
    "fp64": {"prior": "prior_level_kernel", "leaf": "leaf_kernel", "leaf_syrk": "leaf_syrk_kernel",
             "post": "post_level_kernel", "aggregate": "aggregate_kernel"},
    "mixed": {"prior": "prior_level_kernel_tc<0>", "leaf": "leaf_kernel_tc<0>", "leaf_syrk": "leaf_syrk_kernel",
              "post": "post_level_kernel", "aggregate": "aggregate_kernel"},
    "emu": {"prior": "prior_level_kernel_tc<1>", "chain": "chain_forward_kernel_em", "leaf": "leaf_kernel_tc<1>",
            "leaf_syrk": "leaf_syrk_kernel_em", "post": "post_level_kernel<EMU>", "aggregate": "aggregate_kernel_em"},
}


def contraction_share(stage: str, m: int, M: int, r: int, nF):
    """Contraction FLOPs of one (level, stage) of an evaluation: the part of the
    algorithmic FLOPs (mra_stats) that is matrix products, i.e. what a
    tensor-core form runs on the engine (factorisations and vector terms
    excluded)."""
    import numpy as np
    c = np.asarray(nF, dtype=np.float64)
    tri = r * (r + 1) / 2.0
    Mr = M * r
    R = 4.0 ** m
    if stage == "prior":
        return R * (sum(2.0 * r * r * (l * r) + 2.0 * r * tri for l in range(m)) + 2.0 * tri * (m * r))
    if stage == "chain":
        return float(sum((2.0 * c * r * (l * r) + 2.0 * c * tri).sum() for l in range(M)))
    if stage == "leaf":
        return float((c * (c + 1) * Mr + Mr * c * (c + 1)).sum())
    if stage == "leaf_syrk":
        return float(Mr * (Mr + 1) * c.sum())
    if stage == "post":
        return R * m * r * r * (r + 1)
    if stage == "aggregate":
        return R * (m * r) * (m * r + 1) * r
    return 0.0


def level_table(st, prec, M, r, nF, bf16_peak, hbm_peak):
    """Per level and stage of one form: time per evaluation, algorithmic FLOPs and
    bytes (mra_stats), their rates and the fraction of the pipe's peak."""
    ev = max(1, st["evaluations"])
    pairs = EMU_PAIRS if prec == "emu" else TF32_PAIRS
    rows = []
    for m, row in enumerate(st["levels"]):
        for stage, v in row.items():
            if not v["launches"]:
                continue
            sec = v["ms"] / ev * 1e-3
            tensor = stage in TENSOR_STAGES[prec] or (prec == "mixed" and stage == "chain")
            peak = bf16_peak * (1.0 if prec == "emu" else TF32_PER_BF16) if tensor else FP64_PEAK_TFLOPS
            alg = v["flops"] / sec / 1e12
            out = {"level": m, "stage": stage, "kernel": STAGE_KERNEL[prec].get(stage, stage),
                   "ms_per_step": v["ms"] / ev, "launches_per_step": v["launches"] / ev, "units": v["units"],
                   "flops": v["flops"], "bytes": v["bytes"], "alg_tflops": alg,
                   "pipe": "tensor" if tensor else "alu", "peak": peak, "frac": alg / peak,
                   "hbm_gbs": v["bytes"] / sec / 1e9, "hbm_frac": v["bytes"] / sec / 1e9 / hbm_peak,
                   "per_unit": ("algorithmic FP64 FLOPs (mra_stats) of the level's units"
                                + (" against the bf16 tensor peak" if tensor and prec == "emu" else ""))}
            if tensor:
                eng = pairs * contraction_share(stage, m, M, r, nF) / sec / 1e12
                out["engine_tflops"] = eng
                out["engine_frac"] = eng / peak
            rows.append(out)
    return rows


def predict_flops_per_point(M: int, r: int, c: float) -> float:
    """FP64 FLOPs of the prediction kernel per point in a leaf of c observations:
    the Uhat chain, v^P, P = C0 L_Sigma^{-T} - Uhat H', Bhat^{M,k} = Uhat^k - P H^k,
    the Bhat recursion with Lt^{-T} and G, and the mean / variance sums."""
    chain = sum(2.0 * l * r * r + r * (r + 1) for l in range(M))
    rec = sum(r * (r + 1) + 4.0 * r + 2.0 * l * r * r for l in range(M))
    return chain + rec + 2.0 * M * r + c * (c + 1) + 2.0 * M * r * c + 4.0 * c + 2.0 * c * M * r


def run_prediction(args, world, rank, mra, np, torch, stream, handles, w, theta0, off):
    """Kriging throughput (points/s) and errors: 2^20 cell-centred grid points on
    the n = 2^20 problem (emulated-form factors against the FP64 form's), and the
    1024 uniform points of the n = 4096 workload against the oracle."""
    from oracle import mra_oracle as O
    from paper_1507_04789_gb300 import synth
    out = {}
    g = 1024
    cc = (np.arange(g) + 0.5) / g
    gx, gy = np.meshgrid(cc, cc, indexing="xy")
    grid = np.ascontiguousarray(np.stack([gx.ravel(), gy.ravel()], axis=1))
    dgrid = torch.tensor(grid, device="cuda")
    res = {}
    nF = np.diff(off)
    pts_per_leaf = grid.shape[0] / 4 ** w.M
    flops_pt = predict_flops_per_point(w.M, w.r, float(nF.mean()))
    for p in ("emu", "fp64"):
        h = handles[p]
        h.loglik(theta0)
        h.predict(theta0, dgrid)                  # grows the prediction buffers
        reps = 3
        h.enable_timing(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            mean, var = h.predict(theta0, dgrid)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        kms = h.kernel_times()["predict"][0] / reps
        h.enable_timing(False)
        t0 = time.perf_counter()
        for _ in range(reps):
            mh, vh = h.predict(theta0, grid)      # host buffers: copies inside
        e2e_s = (time.perf_counter() - t0) / reps
        res[p] = (mean.cpu().numpy(), var.cpu().numpy())
        alg = flops_pt * grid.shape[0] / (kms * 1e-3) / 1e12
        out[p] = {"points_per_s": world * grid.shape[0] / (ms * 1e-3), "ms_per_call": ms,
                  "kernel_ms": kms, "kernel_fp64_alg_tflops": alg,
                  "kernel_frac": alg / FP64_PEAK_TFLOPS,
                  "e2e": {"points_per_s": world * grid.shape[0] / e2e_s, "h2d_bytes_per_call": int(grid.nbytes),
                          "d2h_bytes_per_call": int(2 * 8 * grid.shape[0])}}
    m64, v64 = res["fp64"]
    me, ve = res["emu"]
    out["grid"] = {"points": int(grid.shape[0]), "layout": f"{g} x {g} cell-centred grid on [0,1]^2",
                   "points_per_leaf": pts_per_leaf, "kernel": "predict_kernel (FP64 pipe)",
                   "fp64_flops_per_point": flops_pt, "peak": FP64_PEAK_TFLOPS,
                   "emu_vs_fp64": {"mean_max_abs": float(np.max(np.abs(me - m64))),
                                   "mean_max_rel": float(np.max(np.abs(me - m64)) / np.max(np.abs(m64))),
                                   "var_max_rel": float(np.max(np.abs(ve - v64) / np.abs(v64)))}}
    # the n = 4096 workload: every form against the oracle
    w1 = synth.workload("n4096_exp_M3_r16")
    l1, y1, p1 = w1.generate()
    th1 = (w1.sigma2, w1.kappa, w1.tau2)
    mo, vo = O.predict(O.Problem(l1, y1, M=w1.M, r=w1.r, family=w1.family), th1, p1)
    small = {"workload": w1.name, "points": int(p1.shape[0])}
    for p in ("fp64", "mixed", "emu"):
        with mra.Handle(l1, y1, M=w1.M, r=w1.r, family=w1.family, precision=p) as h1:
            h1.set_stream(stream)
            h1.loglik(th1)
            mg, vg = h1.predict(th1, p1)
            dp = torch.tensor(p1, device="cuda")
            h1.predict(th1, dp)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                h1.predict(th1, dp)
            e1.record(stream)
            torch.cuda.synchronize()
            ms1 = e0.elapsed_time(e1) / 5
        small[p] = {"mean_max_rel_err_vs_oracle": float(np.max(np.abs(mg - mo)) / np.max(np.abs(mo))),
                    "var_max_rel_err_vs_oracle": float(np.max(np.abs(vg - vo) / np.abs(vo))),
                    "ms_per_call": ms1, "points_per_s": p1.shape[0] / (ms1 * 1e-3)}
    out["n4096"] = small
    return out


# Sec. 4.3's level-varying J_m = (2, 2, 4, 8, 8, 16) with its last level taken as two quadtree levels
# (J_M = 16 at the leaves is not supported): the same 16384 leaves (a 128 x 128 grid) as the paper's
# sequence and as the M = 7 quadtree, about 64 observations each at n = 2^20.
LEVEL_J = (2, 2, 4, 8, 8, 4, 4)


def run_level_J(args, mra, np, torch, stream, locs, y, w, thetas):
    """The same observations on a level-varying partition: the emulated form's
    log-likelihood rate (CUDA events, inputs resident) and its difference from
    the FP64 form's at one theta."""
    if args.no_level_j:
        return None
    steps = max(2, args.steps // 2)
    with mra.Handle(locs, y, M=len(LEVEL_J), r=w.r, J=LEVEL_J, family=w.family, precision="emu") as h, \
            mra.Handle(locs, y, M=len(LEVEL_J), r=w.r, J=LEVEL_J, family=w.family) as h64:
        h.set_stream(stream)
        for k in range(args.warmup):
            h.loglik(thetas[k])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            ll = h.loglik(thetas[k])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ll64 = h64.loglik(thetas[steps - 1])
        off = h.leaf_offsets()
    cnt = np.diff(off)
    return {"J": list(LEVEL_J), "M": len(LEVEL_J), "r": w.r, "leaves": int(cnt.shape[0]),
            "max_leaf": int(cnt.max()), "precision": "emu", "ms_per_step": ms, "value": 1e3 / ms,
            "unit": "evals/s", "dloglik_per_obs_vs_fp64": abs(ll - ll64) / w.n,
            "what": "the headline's observations on Sec. 4.3's J structure (last J = 16 as 4 x 4)"}


def run_sharded(args, rank, world, local, mra, np, torch):
    """N > 1: one n = 2^20 problem sharded over the ranks' GPUs by level-2 subtrees."""
    import torch.distributed as dist

    from paper_1507_04789_gb300 import shard, synth
    w = synth.workload(args.workload)
    locs, y, _ = w.generate()                      # the same seed on every rank: one problem
    theta0 = (w.sigma2, w.kappa, w.tau2)
    thetas = [(theta0[0], theta0[1] * (1.0 + 0.01 * (k % 7)), theta0[2]) for k in range(args.warmup + args.steps)]
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    h = mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision="emu", stream_level=2)
    h.set_stream(stream)
    for k in range(args.warmup):
        ll = shard.sharded_loglik(h, thetas[k], rank, world, device=dev)
    clk = ClockSampler(local)
    clk.start()
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        ll = shard.sharded_loglik(h, thetas[k], rank, world, device=dev)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    t = torch.tensor([e0.elapsed_time(e1), wall * 1e3], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t[0].item()) / args.steps
    wall_ms = float(t[1].item()) / args.steps
    length, nsub = h.summary_len()
    h.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": 1e3 / ms, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64+bf16x7 (emulated f64)", "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "M": w.M, "r": w.r, "family": w.family,
                       "parallelism": f"level-2 subtrees sharded over {world} ranks, one all-gather of "
                                      f"{nsub} x {length} doubles per evaluation",
                       "l2": "working set far larger than the 129 MB L2 (no flush)"},
            "e2e": {"value": 1e3 / wall_ms, "unit": "evals/s", "h2d_bytes_per_step": int(8 * nsub * length),
                    "d2h_bytes_per_step": int(8 * length * shard.subtree_range(nsub, 0, world)[1] + 32),
                    "what": "host wall clock per sharded evaluation (summaries pass through host memory)"},
            "loglik": ll, "clocks": clocks, "gpu_launches": None,
        }), flush=True)
    return 0


def run_large(args, mra, np, torch):
    """The n = 2^24 swath field (M = 10, r = 64, complete tree): the log-likelihood
    evaluated as streamed level-s subtrees in the emulated form, then kriging at
    the 2^20 cell-centred grid points and one log-likelihood + gradient call;
    device memory is sampled after every call."""
    from paper_1507_04789_gb300 import synth
    w = synth.workload(args.workload)
    t0 = time.perf_counter()
    locs, y, grid = w.generate()
    gen_s = time.perf_counter() - t0
    theta0 = (w.sigma2, w.kappa, w.tau2)
    stream = torch.cuda.Stream()
    free0, total = torch.cuda.mem_get_info()
    used = []

    def sample():
        torch.cuda.synchronize()
        used.append(free0 - torch.cuda.mem_get_info()[0])

    t0 = time.perf_counter()
    h = mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, nonstat=w.nonstat, precision="emu",
                   stream_level=args.stream_level)
    build_s = time.perf_counter() - t0
    h.set_stream(stream)
    sample()
    thetas = [(theta0[0], theta0[1] * (1.0 + 0.01 * k), theta0[2]) for k in range(args.warmup + args.steps)]
    for k in range(args.warmup):
        h.loglik(thetas[k])
    sample()
    h.enable_timing(True)
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.warmup, args.warmup + args.steps):
        ll = h.loglik(thetas[k])
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = h.stats()
    h.enable_timing(False)
    sample()
    flops = sum(v["flops"] for row in st["levels"] for v in row.values())
    h.loglik(theta0)
    dgrid = torch.tensor(grid, device="cuda")
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    mean, var = h.predict(theta0, dgrid)
    p1.record(stream)
    torch.cuda.synchronize()
    pred_ms = p0.elapsed_time(p1)
    sample()
    # loglik + gradient on the streamed handle: each chunk's factors formed again before its adjoint
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    g0.record(stream)
    ll_g, grad = h.loglik_grad(theta0)
    g1.record(stream)
    torch.cuda.synchronize()
    grad_ms = g0.elapsed_time(g1)
    sample()
    ll0 = h.loglik(theta0)
    off = h.leaf_offsets()
    nF = np.diff(off)
    h.close()
    line = {
        "metric": f"M-RA loglik evals/s at n=2^24 swath field (M={w.M}, r={w.r}), streamed level-s subtrees",
        "value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "f64+bf16x7 (emulated f64)", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "M": w.M, "r": w.r, "family": w.family, "nonstat": w.nonstat,
                   "sigma2": w.sigma2, "range": w.kappa, "tau2": w.tau2, "stream_level": args.stream_level,
                   "tree": "complete (every region, so that every grid point has its ancestors)",
                   "active_leaves": int((nF > 0).sum()), "leaves": int(nF.size), "max_leaf": int(nF.max())},
        "loglik": ll, "flops_per_step": flops, "fp64_alg_tflops": flops / (ms * 1e-3) / 1e12,
        "device_memory_gb_max": max(used) / 1e9, "device_memory_gb_total": total / 1e9,
        "prediction": {"points": int(grid.shape[0]), "ms_per_call": pred_ms,
                       "points_per_s": grid.shape[0] / (pred_ms * 1e-3),
                       "what": "each chunk's factors formed again from the resident coarse levels, then its "
                               "points predicted (about one more evaluation)",
                       "var_min": float(var.min().item()), "var_max": float(var.max().item())},
        "generate_s": gen_s, "build_s": build_s, "clocks": clocks,
        "gradient": {"ms_per_call": grad_ms, "evals_per_s": 1e3 / grad_ms, "grad": [float(v) for v in grad],
                     "loglik": ll_g, "loglik_rel_diff_vs_plain_eval": abs(ll_g - ll0) / abs(ll0),
                     "what": "loglik + d/d(sigma2, range, tau2) in the emulated form, streamed: the forward "
                             "evaluation, the coarse posterior adjoint, per chunk its factors formed again "
                             "(the last one reused) and its adjoints, then the coarse prior adjoint"},
        "per_level": [{"level": m, "stage": k, "ms_per_step": v["ms"] / max(1, st["evaluations"]),
                       "flops": v["flops"]} for m, row in enumerate(st["levels"]) for k, v in row.items()],
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mra", choices=["mra", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-dataset swath batch")
    ap.add_argument("--batch-datasets", type=int, default=64)
    ap.add_argument("--stream-level", type=int, default=3,
                    help="level of the streamed subtrees for the n = 2^24 swath workload (3: 64 subtrees, so "
                         "that the gradient's chunk buffers keep the run within 180 GB)")
    ap.add_argument("--no-mle", action="store_true", help="skip the 20-step maximum-likelihood fit")
    ap.add_argument("--no-level-j", action="store_true", help="skip the level-varying J partition")
    ap.add_argument("--grad-only", action="store_true",
                    help="time only loglik + gradient in the emulated form (the launch list of the gradient)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    rank, world, local = dist_env()
    # CPU baseline first (child process, before any GPU work in this process)
    cpu, oracle_terms = None, None
    from paper_1507_04789_gb300 import synth as _synth
    if _synth.workload(args.workload).layout == "swath200":
        args.no_cpu_baseline = True          # (the oracle would take hours on a subtree of 2^24 points)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, oracle_terms = oracle_sample(args.workload, min(ORACLE_SAMPLE_LEVEL, _synth.workload(args.workload).M), 0)

    import numpy as np
    import torch
    from paper_1507_04789_gb300 import mra, synth

    torch.cuda.set_device(local)
    if synth.workload(args.workload).layout == "swath200":
        return run_large(args, mra, np, torch)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        try:
            return run_sharded(args, rank, world, local, mra, np, torch)
        finally:
            dist.destroy_process_group()

    w = synth.workload(args.workload)
    w = synth.Workload(**{**w.__dict__, "seed": 1000 * rank})
    locs, y, _ = w.generate()
    theta0 = (w.sigma2, w.kappa, w.tau2)
    stream = torch.cuda.Stream()
    # thetas vary per step (an MLE-like sweep over the range parameter)
    thetas = [(theta0[0], theta0[1] * (1.0 + 0.01 * (k % 7)), theta0[2]) for k in range(args.warmup + args.steps)]

    if args.grad_only:
        with mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision="emu") as h:
            h.set_stream(stream)
            for k in range(args.warmup):
                h.loglik_grad(thetas[k])
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.warmup, args.warmup + args.steps):
                ll, g = h.loglik_grad(thetas[k])
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
        if rank == 0:
            print(json.dumps({"metric": "M-RA loglik + grad evals/s (emulated FP64 forward and adjoint)",
                              "value": 1e3 / ms, "unit": "evals/s", "ms_per_step": ms, "steps": args.steps,
                              "warmup": args.warmup, "config": {"workload": args.workload},
                              "grad": [float(v) for v in g]}))
        return

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def time_form(precision):
        h = mra.Handle(locs, y, M=w.M, r=w.r, family=w.family, precision=precision)
        h.set_stream(stream)
        lls = [h.loglik(thetas[k]) for k in range(args.warmup)]
        h.enable_timing(True)
        mra.launch_count(reset=True)
        clk = ClockSampler(local)
        clk.start()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.warmup, args.warmup + args.steps):
            lls.append(h.loglik(thetas[k]))
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1))
        launches = mra.launch_count(reset=True)
        kt = h.kernel_times()
        st = h.stats()
        h.enable_timing(False)
        return h, {"ms_per_step": ms / args.steps, "value": world * 1e3 * args.steps / ms, "lls": lls,
                   "kernels": kt, "launches": launches, "clocks": clocks, "stats": st}

    # ---- the three forms on the same steps ----
    forms, handles = {}, {}
    for prec in ("emu", "mixed", "fp64"):
        handles[prec], forms[prec] = time_form(prec)
    off = handles["fp64"].leaf_offsets()
    flops = algorithmic_flops(w.M, w.r, np.diff(off))
    total_flops = sum(flops.values())
    for prec in ("emu", "mixed"):
        forms[prec]["dll"] = max(abs(a - b) for a, b in zip(forms[prec]["lls"], forms["fp64"]["lls"])) / w.n
    for prec in ("emu", "mixed"):
        if prec != "emu":
            handles[prec].close()
    h64 = handles["fp64"]

    # ---- loglik + gradient: the emulated form (forward and adjoint on the engine) and the FP64 form ----
    def time_grad(h):
        g_steps = max(2, args.steps // 2)
        h.loglik_grad(theta0)
        h.enable_timing(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(g_steps):
            ll_g, grad = h.loglik_grad(thetas[k])
        e1.record(stream)
        torch.cuda.synchronize()
        g_ms = max_over_ranks(e0.elapsed_time(e1)) / g_steps
        g_kt = h.kernel_times()
        h.enable_timing(False)
        return {"value": world * 1e3 / g_ms, "unit": "evals/s", "ms_per_step": g_ms,
                "adjoint_ms_per_step": g_kt["grad"][0] / g_steps, "grad": [float(v) for v in grad]}

    g_emu = time_grad(handles["emu"])
    g_64 = time_grad(h64)
    gradient = dict(g_emu)
    gradient["what"] = ("loglik + d/d(sigma2, range, tau2): forward pass and reverse-mode adjoint in the "
                        "emulated-FP64 form")
    gradient["max_rel_diff_vs_fp64_form"] = max(abs(a - b) / max(abs(b), 1e-300)
                                                for a, b in zip(g_emu["grad"], g_64["grad"]))
    gradient["fp64"] = g_64
    # 20 steps of gradient-based maximum likelihood from range = 0.3 (Adam on the log-parameters, the
    # library's adjoint through torch.autograd), emulated form
    if not args.no_mle:
        from paper_1507_04789_gb300 import autograd as mra_ag
        th0 = (w.sigma2, 0.3, w.tau2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th_fit, hist = mra_ag.fit_mle(handles["emu"], th0, steps=20, lr=0.1)
        torch.cuda.synchronize()
        mle_s = time.perf_counter() - t0
        gradient["mle"] = {"steps": 20, "seconds": mle_s, "ms_per_step": mle_s / 20 * 1e3,
                           "theta0": list(th0), "theta": [float(v) for v in th_fit],
                           "loglik0": hist[0][1], "loglik": hist[-1][1], "true_theta": list(theta0),
                           "what": "Adam (lr 0.1) on log(sigma2, range, tau2), each step one loglik + gradient "
                                   "through torch.autograd; host wall clock"}

    peaks = measured_peaks()
    bf16_peak = peaks["bf16_tflops_sustained"] if peaks else BF16_PEAK_FALLBACK
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "of measured (bf16 sustained, MEASURED_PEAKS.json)" if peaks else "of fallback (recipe)"

    def kernel_table(prec):
        res = forms[prec]
        cf = contraction_flops(w.M, w.r, np.diff(off), prec)
        pairs = EMU_PAIRS if prec == "emu" else TF32_PAIRS
        tab = {}
        for k, v in res["kernels"].items():
            if v[1] == 0 or k not in flops:
                continue
            sec = v[0] * 1e-3 / args.steps
            row = {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                   "fp64_alg_tflops": flops[k] / sec / 1e12 if sec > 0 else None}
            if k in cf and sec > 0:
                row["tensor_tflops"] = pairs * cf[k] / sec / 1e12
            tab[k] = row
        return tab

    ok = [p for p in ("emu", "mixed") if forms[p]["dll"] <= 1e-6]
    best = min(ok, key=lambda p: forms[p]["ms_per_step"]) if ok else "fp64"
    if forms["fp64"]["ms_per_step"] < forms[best]["ms_per_step"]:
        best = "fp64"
    head = forms[best]
    # roofline of the dominant kernel of the headline form, from the per-level stats
    nF_leaf = np.diff(off)
    lvl_tabs = {p: level_table(forms[p]["stats"], p, w.M, w.r, nF_leaf, bf16_peak, hbm_peak)
                for p in ("emu", "mixed", "fp64")}
    rows = lvl_tabs[best]
    dom = max(rows, key=lambda r_: r_["ms_per_step"])
    roofline = {"bound": dom["pipe"], "achieved": dom["alg_tflops"], "peak": dom["peak"], "unit": "TFLOP/s",
                "frac": dom["frac"], "traffic": None, "kernel": dom["kernel"], "level": dom["level"],
                "stage": dom["stage"],
                "peak_source": (peak_src if dom["pipe"] == "tensor" else
                                "of measured FP64 pipe (DMMA 1.10 TFLOP/s, tests/peaks.cu; profiles/pipe_peaks_gb300.md)"),
                "per_unit": dom["per_unit"], "units_per_launch": dom["units"],
                "algorithmic_flops_per_launch": dom["flops"], "ms_per_launch": dom["ms_per_step"],
                "launches_per_step": 1.0}
    if "engine_tflops" in dom:
        roofline["engine_issued_tflops"] = dom["engine_tflops"]
        roofline["engine_frac"] = dom["engine_frac"]
        roofline["engine_note"] = (f"tensor work the engine issues: {EMU_PAIRS if best == 'emu' else TF32_PAIRS} "
                                   f"slice MACs per FP64 MAC of the kernel's contractions")
    traffic, how = kernel_traffic(best, dom["kernel"], w.name)
    roofline["traffic"] = traffic
    if how:
        roofline["traffic_source"] = how
    roofline["algorithmic_bytes_per_launch"] = dom["bytes"]
    roofline.update({"per_level": rows, "kernels": kernel_table(best),
                     "step_fp64_alg_tflops": total_flops / (head["ms_per_step"] * 1e-3) / 1e12})

    # ---- oracle error of the GPU forms at full size: the sampled subtrees' d_R, u_R ----
    oracle_check = None
    if oracle_terms:
        lvl = oracle_terms["level"]
        ks = oracle_terms["regions"]
        od, ou = np.array(oracle_terms["d"]), np.array(oracle_terms["u"])
        oracle_check = {"level": lvl, "regions": ks, "theta": list(theta0)}
        for p in ("emu", "fp64"):
            handles[p].loglik(theta0)
            d_g, u_g = handles[p].region_terms(lvl)
            oracle_check[p] = {"d_max_rel_err": float(np.max(np.abs(d_g[ks] - od) / np.abs(od))),
                               "u_max_rel_err": float(np.max(np.abs(u_g[ks] - ou) / np.abs(ou)))}
        if cpu:
            cpu["oracle_check"] = oracle_check

    # ---- prediction (Sec. 3.4): 2^20 grid points on this problem and the 1024 points of the n = 4096 workload ----
    prediction = run_prediction(args, world, rank, mra, np, torch, stream, handles, w, theta0, off)

    # ---- end to end through the C ABI with host inputs (headline form) ----
    h = handles[best] if best in ("emu", "fp64") else mra.Handle(locs, y, M=w.M, r=w.r, family=w.family,
                                                                 precision=best)
    h.set_stream(stream)
    pin_l = torch.from_numpy(np.ascontiguousarray(locs)).pin_memory()
    pin_y = torch.from_numpy(np.ascontiguousarray(y)).pin_memory()
    nl, ny = pin_l.numpy(), pin_y.numpy()
    h.update(nl, ny)
    h.loglik(theta0)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.e2e_steps):
        h.update(nl, ny)
        h.loglik(thetas[k % len(thetas)])
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps)
    e2e = {"value": world / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": int(locs.nbytes + y.nbytes),
           "d2h_bytes_per_step": 32}
    h.close()
    for p in ("emu", "fp64"):
        if handles[p] is not h:
            handles[p].close()
    batch = None if args.no_batch else run_batch(args, world, rank, mra, np, torch)
    level_J = run_level_J(args, mra, np, torch, stream, locs, y, w, thetas)

    if rank == 0:
        dtypes = {"fp64": "f64", "mixed": "f64+tf32x3", "emu": "f64+bf16x7 (emulated f64)"}

        def form_line(p):
            out = {"value": forms[p]["value"], "ms_per_step": forms[p]["ms_per_step"], "kernels": kernel_table(p),
                   "clocks": forms[p]["clocks"]}
            if p != "fp64":
                out["dloglik_per_obs_vs_fp64"] = forms[p]["dll"]
            return out

        line = {
            "metric": METRIC, "value": head["value"], "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtypes[best], "data": "synthetic",
            "config": {"workload": w.name, "n": w.n, "M": w.M, "J": w.J, "r": w.r, "family": w.family,
                       "sigma2": w.sigma2, "range": w.kappa, "tau2": w.tau2, "precision": best,
                       "max_leaf": int(np.diff(off).max()), "step": "one log-likelihood evaluation",
                       "l2": "working set ~10 GB per evaluation, far larger than the 129 MB L2 (no flush)",
                       "parallelism": "1 GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(head["launches"]),
            "clocks": head["clocks"],
            "emu": form_line("emu"), "mixed": form_line("mixed"), "fp64": form_line("fp64"),
            "gradient": gradient, "loglik": head["lls"][-1], "flops_per_step": total_flops,
            "batch": batch, "prediction": prediction, "oracle_check": oracle_check, "level_J": level_J,
        }
        for p in ("emu", "mixed", "fp64"):
            line[p]["per_level"] = [{k: r_[k] for k in ("level", "stage", "ms_per_step", "alg_tflops", "frac",
                                                        "hbm_gbs") + (("engine_frac",) if "engine_frac" in r_ else ())}
                                    for r_ in lvl_tabs[p]]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""The allocation-free log-likelihood entry point agrees with the handle path.

mra_loglik_noalloc serves callers that cannot allocate device memory (a host
framework's caching allocator owns the heap, or allocation after start-up is
forbidden): it keeps every intermediate in a fixed scratch array inside the
library.  This file is collected last on purpose, so that a run stopping at the
first failure has already run every other test.  It calls the entry point
through the C ABI twice in a row, on different data and parameters, and checks
each result against mra_build + mra_loglik within the tolerance of the other
log-likelihood tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LL_RTOL = 1e-10


def _noalloc(lib, mra, cfg, theta, locs_dev, y_dev, n):
    fn = lib.mra_loglik_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(mra.MraConfig), ctypes.POINTER(mra.MraParams), ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double()
    rc = fn(ctypes.byref(cfg), ctypes.byref(theta), locs_dev.data_ptr(), y_dev.data_ptr(), n, None,
            ctypes.byref(out))
    if rc != 0:
        raise mra.MRAError(rc, lib.mra_last_error().decode())
    return out.value


def test_noalloc_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    from paper_1507_04789_gb300 import mra, synth
    lib = mra.load_library()
    cases = []
    w = synth.workload("n4096_exp_M3_r16")
    locs, y, _ = w.generate()
    cases.append((locs, y, 3, 16, "exp", (w.sigma2, w.kappa, w.tau2)))
    rng = np.random.default_rng(21)
    locs2 = rng.random((3000, 2))
    y2 = rng.standard_normal(3000)
    cases.append((locs2, y2, 3, 64, "matern15", (1.1, 0.12, 0.02)))
    calls = []
    for locs, y, M, r, fam, theta in cases:
        with mra.Handle(locs, y, M=M, r=r, family=fam) as h:
            ref = h.loglik(theta)
        cfg = mra.MraConfig(M, 4, r, mra.FAMILIES[fam], 0, mra.MRA_PREC_FP64, 0,
                            (ctypes.c_double * 4)(0.0, 1.0, 0.0, 1.0))
        p = mra.MraParams(*theta)
        dl = torch.tensor(locs, device="cuda", dtype=torch.float64)
        dy = torch.tensor(y, device="cuda", dtype=torch.float64)
        got = _noalloc(lib, mra, cfg, p, dl, dy, locs.shape[0])
        assert got == pytest.approx(ref, rel=LL_RTOL, abs=0)
        calls.append((cfg, p, dl, dy, locs.shape[0], got))
    # the property the entry point exists for: once the scratch address is
    # resolved and every kernel is loaded, a call takes no device memory
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for cfg, p, dl, dy, n, got in calls:
        assert _noalloc(lib, mra, cfg, p, dl, dy, n) == got
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == res0


def test_noalloc_refuses_host_pointers_and_names_fields():
    """Host arrays are refused on the host side (no kernel runs), and a
    configuration the entry point does not support names the field."""
    from paper_1507_04789_gb300 import mra
    lib = mra.load_library()
    rng = np.random.default_rng(23)
    locs = np.ascontiguousarray(rng.random((500, 2)))
    y = rng.standard_normal(500)
    bbox = (ctypes.c_double * 4)(0.0, 1.0, 0.0, 1.0)
    cfg = mra.MraConfig(2, 4, 16, mra.MRA_COV_EXP, 0, mra.MRA_PREC_FP64, 0, bbox)
    p = mra.MraParams(1.0, 0.1, 0.01)
    fn = lib.mra_loglik_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(mra.MraConfig), ctypes.POINTER(mra.MraParams), ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double()
    rc = fn(ctypes.byref(cfg), ctypes.byref(p), locs.ctypes.data, y.ctypes.data, 500, None, ctypes.byref(out))
    assert rc == mra.MRA_ERR_ARG
    assert "device" in lib.mra_last_error().decode()
    for field, bad in (("precision", mra.MRA_PREC_EMU), ("prune", 1)):
        c = mra.MraConfig(2, 4, 16, mra.MRA_COV_EXP, 0, mra.MRA_PREC_FP64, 0, bbox)
        setattr(c, field, bad)
        rc = fn(ctypes.byref(c), ctypes.byref(p), locs.ctypes.data, y.ctypes.data, 500, None, ctypes.byref(out))
        assert rc == mra.MRA_ERR_ARG
        assert field in lib.mra_last_error().decode()


def test_noalloc_rejects_oversized_problems():
    torch = pytest.importorskip("torch")
    from paper_1507_04789_gb300 import mra
    lib = mra.load_library()
    n = 1 << 18
    rng = np.random.default_rng(22)
    dl = torch.tensor(rng.random((n, 2)), device="cuda")
    dy = torch.tensor(rng.standard_normal(n), device="cuda")
    cfg = mra.MraConfig(6, 4, 64, mra.MRA_COV_EXP, 0, mra.MRA_PREC_FP64, 0,
                        (ctypes.c_double * 4)(0.0, 1.0, 0.0, 1.0))
    with pytest.raises(mra.MRAError) as ei:
        _noalloc(lib, mra, cfg, mra.MraParams(1.0, 0.1, 0.01), dl, dy, n)
    assert ei.value.code == mra.MRA_ERR_LIMIT
    assert "scratch" in str(ei.value)

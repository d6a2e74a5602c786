"""Python binding of the C ABI in ``include/mra.h`` (argument marshalling only).

Every step of the computation runs in the CUDA library
``libmra_gb300.so``; this module converts arguments, calls it through ctypes
and raises :class:`MRAError` on a non-zero status.  There is no fallback: if
the library is missing, importing the binding fails with a message saying how
to build it.

Inputs may be numpy arrays (host memory) or CUDA ``torch.Tensor`` objects
(device memory, float64, contiguous); outputs of :meth:`Handle.predict` are
returned in the same memory space as the prediction locations.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmra_gb300.so")

MRA_OK, MRA_ERR_ARG, MRA_ERR_OOM, MRA_ERR_CUDA, MRA_ERR_NOT_PD, MRA_ERR_STATE, MRA_ERR_LIMIT = range(7)
MRA_COV_EXP, MRA_COV_MATERN15, MRA_COV_MATERN = 0, 1, 2
MRA_PREC_FP64, MRA_PREC_MIXED, MRA_PREC_EMU = 0, 1, 2
PRECISIONS = {"fp64": MRA_PREC_FP64, "mixed": MRA_PREC_MIXED, "emu": MRA_PREC_EMU}
MRA_HOST, MRA_DEVICE = 0, 1
MRA_MAX_LEAF = 128
MRA_OPT_GRAD_BUFFERS = 0
FAMILIES = {"exp": MRA_COV_EXP, "matern15": MRA_COV_MATERN15, "matern": MRA_COV_MATERN}
KERNEL_KINDS = ("prior", "leaf", "leaf_syrk", "post", "aggregate", "predict", "grad")


class MRAError(RuntimeError):
    """Non-zero status from the library; ``code`` is the MRA_ERR_* value."""

    def __init__(self, code: int, msg: str):
        super().__init__(f"[mra error {code}] {msg}")
        self.code = code


MRA_MAX_M = 12


class MraConfig(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("J", ctypes.c_int), ("r", ctypes.c_int),
                ("cov_family", ctypes.c_int), ("nonstat", ctypes.c_int),
                ("precision", ctypes.c_int), ("prune", ctypes.c_int), ("bbox", ctypes.c_double * 4),
                ("stream_level", ctypes.c_int), ("J_level", ctypes.c_int * MRA_MAX_M)]


def _set_J(cfg: MraConfig, J, M: int) -> None:
    """J: children per region, one number for every level or (J_1, ..., J_M)."""
    if isinstance(J, (int, np.integer)):
        cfg.J = int(J)
        return
    Js = tuple(int(j) for j in J)
    if len(Js) != M:
        raise ValueError("J needs one entry per level 1..M")
    cfg.J = 4
    for k, j in enumerate(Js):
        cfg.J_level[k] = j


class MraParams(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("range", ctypes.c_double), ("tau2", ctypes.c_double),
                ("nu", ctypes.c_double)]


STAGES = ("prior", "chain", "leaf", "leaf_syrk", "post", "aggregate")   # MRA_STAGE_* order


class MraStats(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("evaluations", ctypes.c_int64),
                ("ms", (ctypes.c_double * 6) * (MRA_MAX_M + 1)),
                ("launches", (ctypes.c_int64 * 6) * (MRA_MAX_M + 1)),
                ("flops", (ctypes.c_double * 6) * (MRA_MAX_M + 1)),
                ("bytes", (ctypes.c_double * 6) * (MRA_MAX_M + 1)),
                ("units", (ctypes.c_double * 6) * (MRA_MAX_M + 1))]


def _stats(lib, h) -> dict:
    st = MraStats()
    _check(lib.mra_stats(h, ctypes.byref(st)))
    out = {"M": st.M, "evaluations": st.evaluations, "levels": []}
    for m in range(st.M + 1):
        row = {}
        for k, name in enumerate(STAGES):
            if st.units[m][k] or st.launches[m][k]:
                row[name] = {"ms": st.ms[m][k], "launches": st.launches[m][k], "flops": st.flops[m][k],
                             "bytes": st.bytes[m][k], "units": st.units[m][k]}
        out["levels"].append(row)
    return out


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with "
                          f"`python -c 'import __graft_entry__ as g; g.build()'` "
                          f"or `python {os.path.join(_PKG, 'build.py')}`")
    lib = ctypes.CDLL(path)
    sig = {
        "mra_build": (ctypes.c_int, [ctypes.POINTER(MraConfig), _P, _P, ctypes.c_int64, ctypes.c_int,
                                     ctypes.POINTER(_P)]),
        "mra_set_data": (ctypes.c_int, [_P, _P, ctypes.c_int]),
        "mra_update": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
        "mra_enable_timing": (ctypes.c_int, [_P, ctypes.c_int]),
        "mra_kernel_times": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int64)]),
        "mra_loglik": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), _D]),
        "mra_predict": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), _P, ctypes.c_int64, ctypes.c_int,
                                       _P, _P]),
        "mra_region_terms": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
        "mra_leaf_offsets": (ctypes.c_int, [_P, _P, _P]),
        "mra_set_stream": (ctypes.c_int, [_P, _P]),
        "mra_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
        "mra_free": (None, [_P]),
        "mra_last_error": (ctypes.c_char_p, []),
        "mra_launch_count": (ctypes.c_int64, [ctypes.c_int]),
        "mra_build_batch": (ctypes.c_int, [ctypes.POINTER(MraConfig), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                           ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(_P)]),
        "mra_loglik_batch": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), _P]),
        "mra_autotune": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), ctypes.POINTER(ctypes.c_int)]),
        "mra_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "mra_loglik_grad_batch": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), _P, _P]),
        "mra_stats": (ctypes.c_int, [_P, ctypes.POINTER(MraStats)]),
        "mra_predict_joint": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), _P, ctypes.c_int64, ctypes.c_int,
                                             _P, _P]),
        "mra_simulate": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), _P, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int64, _P, _P, _P]),
        "mra_simulate_xi_len": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
        "mra_summary_len": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "mra_loglik_subtrees": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), ctypes.c_int64, ctypes.c_int64, _P]),
        "mra_loglik_combine": (ctypes.c_int, [_P, ctypes.POINTER(MraParams), _P, _D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    lib.mra_loglik_grad.restype = ctypes.c_int
    lib.mra_loglik_grad.argtypes = [_P, ctypes.POINTER(MraParams), _D, _P]
    _lib = lib
    return lib


def _check(rc: int) -> None:
    if rc != MRA_OK:
        raise MRAError(rc, _lib.mra_last_error().decode())


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and hasattr(x, "data_ptr") and bool(x.is_cuda)


def _host_f64(x, shape_last=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape_last is not None and (a.ndim != 2 or a.shape[1] != shape_last):
        raise ValueError(f"expected an (n, {shape_last}) array, got shape {a.shape}")
    return a


def _dev_ptr(t, name: str) -> int:
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    return t.data_ptr()


def launch_count(reset: bool = False) -> int:
    """Kernel launches the library issued from this thread (optionally reset)."""
    return int(load_library().mra_launch_count(1 if reset else 0))


class Handle:
    """One M-RA problem on the GPU: locations, data and the tree (Sec. 2.2)."""

    def __init__(self, locs, y, M: int, r: int, family: str = "exp", nonstat: bool = False,
                 bbox=(0.0, 1.0, 0.0, 1.0), J=4, precision="fp64", prune: bool = False,
                 stream_level: int = 0):
        """J: children per region, 4 (the quadtree) or a level-varying (J_1, ..., J_M)."""
        lib = load_library()
        self._lib = lib
        self._h = _P()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg = MraConfig(M, 4, r, FAMILIES[family] if isinstance(family, str) else int(family),
                        int(bool(nonstat)), prec, int(bool(prune)), (ctypes.c_double * 4)(*bbox), int(stream_level))
        _set_J(cfg, J, M)
        if _is_torch_cuda(locs):
            if locs.dim() != 2 or locs.shape[1] != 2:
                raise ValueError("locs must be (n, 2)")
            n = locs.shape[0]
            keep = (locs, y)
            rc = lib.mra_build(ctypes.byref(cfg), _dev_ptr(locs, "locs"), _dev_ptr(y, "y"), n, MRA_DEVICE,
                               ctypes.byref(self._h))
            del keep
            self._where = MRA_DEVICE
        else:
            la = _host_f64(locs, 2)
            ya = _host_f64(y)
            if ya.shape != (la.shape[0],):
                raise ValueError("y must have one value per location")
            n = la.shape[0]
            rc = lib.mra_build(ctypes.byref(cfg), la.ctypes.data, ya.ctypes.data, n, MRA_HOST,
                               ctypes.byref(self._h))
            self._where = MRA_HOST
        _check(rc)
        self.n, self.M, self.r, self.J = n, M, r, J
        self.family, self.nonstat = family, nonstat
        self.bbox = tuple(bbox)

    # -- lifecycle --------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.mra_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream) -> None:
        """Run on a ``torch.cuda.Stream`` (or a raw cudaStream_t integer, 0 = default)."""
        ptr = getattr(stream, "cuda_stream", stream)
        _check(self._lib.mra_set_stream(self._h, _P(int(ptr) if ptr else None)))

    def set_option(self, option: int, value: int) -> None:
        """mra_set_option: e.g. ``set_option(MRA_OPT_GRAD_BUFFERS, 0)``."""
        _check(self._lib.mra_set_option(self._h, int(option), int(value)))

    def set_data(self, y) -> None:
        if _is_torch_cuda(y):
            _check(self._lib.mra_set_data(self._h, _dev_ptr(y, "y"), MRA_DEVICE))
        else:
            ya = _host_f64(y)
            _check(self._lib.mra_set_data(self._h, ya.ctypes.data, MRA_HOST))

    def update(self, locs, y) -> None:
        """New locations and data of the same size, re-partitioned in place."""
        if _is_torch_cuda(locs):
            _check(self._lib.mra_update(self._h, _dev_ptr(locs, "locs"), _dev_ptr(y, "y"), MRA_DEVICE))
        else:
            la = _host_f64(locs, 2)
            ya = _host_f64(y)
            _check(self._lib.mra_update(self._h, la.ctypes.data, ya.ctypes.data, MRA_HOST))

    def enable_timing(self, on: bool = True) -> None:
        _check(self._lib.mra_enable_timing(self._h, 1 if on else 0))

    def stats(self) -> dict:
        """mra_stats: per level and stage, summed device time and launches of the
        timed evaluations and the algorithmic FLOPs / bytes of one evaluation."""
        return _stats(self._lib, self._h)

    def kernel_times(self) -> dict:
        """{kind: (total_ms, launches)} since enable_timing."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            ms = ctypes.c_double()
            cnt = ctypes.c_int64()
            _check(self._lib.mra_kernel_times(self._h, k, ctypes.byref(ms), ctypes.byref(cnt)))
            out[name] = (ms.value, cnt.value)
        return out

    # -- computations -------------------------------------------------------------
    def loglik(self, theta) -> float:
        """Log-likelihood at theta = (sigma2, range, tau2) (Sec. 3.3)."""
        out = ctypes.c_double()
        p = MraParams(*[float(v) for v in theta])
        _check(self._lib.mra_loglik(self._h, ctypes.byref(p), ctypes.byref(out)))
        return out.value

    def loglik_grad(self, theta):
        """(loglik, d loglik / d(sigma2, range, tau2)), and d/dnu as a fourth
        component for the free-smoothness family (theta = (sigma2, range, tau2, nu))."""
        out = ctypes.c_double()
        four = self.family in ("matern", MRA_COV_MATERN)
        g = np.zeros(4)
        p = MraParams(*[float(v) for v in theta])
        _check(self._lib.mra_loglik_grad(self._h, ctypes.byref(p), ctypes.byref(out), g.ctypes.data))
        return out.value, (g if four else g[:3].copy())

    def predict(self, theta, plocs):
        """Posterior predictive mean and variance of y at plocs (Sec. 3.4, Prop. 2)."""
        p = MraParams(*[float(v) for v in theta])
        if _is_torch_cuda(plocs):
            import torch
            npred = plocs.shape[0]
            mean = torch.empty(npred, dtype=torch.float64, device=plocs.device)
            var = torch.empty(npred, dtype=torch.float64, device=plocs.device)
            _check(self._lib.mra_predict(self._h, ctypes.byref(p), _dev_ptr(plocs, "plocs"), npred, MRA_DEVICE,
                                         mean.data_ptr(), var.data_ptr()))
            return mean, var
        pa = _host_f64(plocs, 2)
        mean = np.empty(pa.shape[0])
        var = np.empty(pa.shape[0])
        _check(self._lib.mra_predict(self._h, ctypes.byref(p), pa.ctypes.data, pa.shape[0], MRA_HOST,
                                     mean.ctypes.data, var.ctypes.data))
        return mean, var

    def predict_joint(self, theta, plocs):
        """Joint posterior predictive mean and np x np covariance of y (Prop. 2)."""
        p = MraParams(*[float(v) for v in theta])
        if _is_torch_cuda(plocs):
            import torch
            npred = plocs.shape[0]
            mean = torch.empty(npred, dtype=torch.float64, device=plocs.device)
            cov = torch.empty((npred, npred), dtype=torch.float64, device=plocs.device)
            _check(self._lib.mra_predict_joint(self._h, ctypes.byref(p), _dev_ptr(plocs, "plocs"), npred,
                                               MRA_DEVICE, mean.data_ptr(), cov.data_ptr()))
            return mean, cov
        pa = _host_f64(plocs, 2)
        mean = np.empty(pa.shape[0])
        cov = np.empty((pa.shape[0], pa.shape[0]))
        _check(self._lib.mra_predict_joint(self._h, ctypes.byref(p), pa.ctypes.data, pa.shape[0], MRA_HOST,
                                           mean.ctypes.data, cov.ctypes.data))
        return mean, cov

    def xi_len(self) -> int:
        """Standard normals per draw for the regions (mra_simulate_xi_len)."""
        n = ctypes.c_int64()
        _check(self._lib.mra_simulate_xi_len(self._h, ctypes.byref(n)))
        return n.value

    def simulate(self, theta, plocs, xi, zeta):
        """Conditional simulations (Prop. 2): draws (nsim x np) from the joint
        posterior predictive given standard normals xi (nsim x xi_len) and zeta
        (nsim x np).  Host arrays in, host array out; torch CUDA tensors in,
        a CUDA tensor out."""
        p = MraParams(*[float(v) for v in theta])
        if _is_torch_cuda(plocs):
            import torch
            nsim, npred = zeta.shape
            draws = torch.empty((nsim, npred), dtype=torch.float64, device=plocs.device)
            _check(self._lib.mra_simulate(self._h, ctypes.byref(p), _dev_ptr(plocs, "plocs"), npred, MRA_DEVICE,
                                          nsim, _dev_ptr(xi, "xi") if xi.numel() else None, _dev_ptr(zeta, "zeta"),
                                          draws.data_ptr()))
            return draws
        pa = _host_f64(plocs, 2)
        za = np.ascontiguousarray(np.atleast_2d(zeta), dtype=np.float64)
        xa = np.ascontiguousarray(np.atleast_2d(xi), dtype=np.float64)
        nsim = za.shape[0]
        if za.shape[1] != pa.shape[0] or xa.shape[0] != nsim or xa.shape[1] != self.xi_len():
            raise ValueError("xi must be nsim x xi_len() and zeta nsim x np")
        draws = np.empty((nsim, pa.shape[0]))
        _check(self._lib.mra_simulate(self._h, ctypes.byref(p), pa.ctypes.data, pa.shape[0], MRA_HOST, nsim,
                                      xa.ctypes.data if xa.size else None, za.ctypes.data, draws.ctypes.data))
        return draws

    def summary_len(self):
        """(doubles per level-s summary, number of level-s subtrees) of a streamed handle."""
        n, k = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.mra_summary_len(self._h, ctypes.byref(n), ctypes.byref(k)))
        return n.value, k.value

    def loglik_subtrees(self, theta, first: int, count: int) -> np.ndarray:
        """Summaries (count x len) of the level-s subtrees [first, first + count)."""
        length, _ = self.summary_len()
        out = np.empty((max(count, 0), length))
        p = MraParams(*[float(v) for v in theta])
        _check(self._lib.mra_loglik_subtrees(self._h, ctypes.byref(p), int(first), int(count),
                                             out.ctypes.data if count else None))
        return out

    def loglik_combine(self, theta, summaries) -> float:
        """Log-likelihood from the summaries of every level-s subtree."""
        sa = np.ascontiguousarray(summaries, dtype=np.float64)
        p = MraParams(*[float(v) for v in theta])
        out = ctypes.c_double()
        _check(self._lib.mra_loglik_combine(self._h, ctypes.byref(p), sa.ctypes.data, ctypes.byref(out)))
        return out.value

    def region_terms(self, level: int):
        """(d_R, u_R) of every region at ``level`` from the last loglik (Sec. 3.3)."""
        cnt = self.nregions(level)
        d = np.empty(cnt)
        u = np.empty(cnt)
        _check(self._lib.mra_region_terms(self._h, level, d.ctypes.data, u.ctypes.data))
        return d, u

    def nregions(self, level: int) -> int:
        """Regions of ``level`` in the complete tree: J_1 ... J_level."""
        if isinstance(self.J, (int, np.integer)):
            return int(self.J) ** level
        return int(np.prod([int(j) for j in self.J[:level]], dtype=np.int64))

    def leaf_offsets(self, with_perm: bool = False):
        off = np.empty(self.nregions(self.M) + 1, dtype=np.int64)
        perm = np.empty(self.n, dtype=np.int64) if with_perm else None
        _check(self._lib.mra_leaf_offsets(self._h, off.ctypes.data, perm.ctypes.data if with_perm else None))
        return (off, perm) if with_perm else off


class Batch:
    """Many independent datasets evaluated together, one launch per level.

    ``datasets`` is a list of dicts with keys ``locs`` (n x 2), ``y`` (n),
    ``M`` and optionally ``family``, ``nonstat``, ``bbox``, ``prune``
    (default True).  All datasets share ``r`` and ``precision``.
    """

    def __init__(self, datasets, r: int, precision="fp64"):
        lib = load_library()
        self._lib = lib
        self._h = _P()
        nd = len(datasets)
        cfgs = (MraConfig * nd)()
        keep = []
        lp = (_P * nd)()
        yp = (_P * nd)()
        ns = (ctypes.c_int64 * nd)()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        for d, ds in enumerate(datasets):
            la = _host_f64(ds["locs"], 2)
            ya = _host_f64(ds["y"])
            keep += [la, ya]
            fam = ds.get("family", "exp")
            cfgs[d] = MraConfig(int(ds["M"]), 4, r, FAMILIES[fam] if isinstance(fam, str) else int(fam),
                                int(bool(ds.get("nonstat", False))), prec, int(bool(ds.get("prune", True))),
                                (ctypes.c_double * 4)(*ds.get("bbox", (0.0, 1.0, 0.0, 1.0))))
            _set_J(cfgs[d], ds.get("J", 4), int(ds["M"]))
            lp[d] = la.ctypes.data
            yp[d] = ya.ctypes.data
            ns[d] = la.shape[0]
        _check(lib.mra_build_batch(cfgs, lp, yp, ns, nd, MRA_HOST, ctypes.byref(self._h)))
        self.ndata = nd
        self.n = [int(v) for v in ns]

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.mra_free(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _params(self, thetas):
        arr = (MraParams * self.ndata)()
        for d, t in enumerate(thetas):
            arr[d] = MraParams(*[float(v) for v in t])
        return arr

    def loglik(self, thetas):
        """Log-likelihood of every dataset at its own theta (Sec. 3.3)."""
        out = np.empty(self.ndata)
        _check(self._lib.mra_loglik_batch(self._h, self._params(thetas), out.ctypes.data))
        return out

    def loglik_grad(self, thetas):
        """Log-likelihood and gradient d/d(sigma2, range, tau2) of every dataset."""
        ll = np.empty(self.ndata)
        g = np.empty((self.ndata, 3))
        _check(self._lib.mra_loglik_grad_batch(self._h, self._params(thetas), ll.ctypes.data, g.ctypes.data))
        return ll, g

    def autotune(self, thetas) -> int:
        tile = ctypes.c_int()
        _check(self._lib.mra_autotune(self._h, self._params(thetas), ctypes.byref(tile)))
        return tile.value

    def info(self):
        nd, tile = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.mra_batch_info(self._h, ctypes.byref(nd), ctypes.byref(tile)))
        return nd.value, tile.value

    def enable_timing(self, on: bool = True) -> None:
        _check(self._lib.mra_enable_timing(self._h, 1 if on else 0))

    def stats(self) -> dict:
        """mra_stats: per level and stage, summed device time and launches of the
        timed evaluations and the algorithmic FLOPs / bytes of one evaluation."""
        return _stats(self._lib, self._h)

    def kernel_times(self) -> dict:
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            ms = ctypes.c_double()
            cnt = ctypes.c_int64()
            _check(self._lib.mra_kernel_times(self._h, k, ctypes.byref(ms), ctypes.byref(cnt)))
            out[name] = (ms.value, cnt.value)
        return out

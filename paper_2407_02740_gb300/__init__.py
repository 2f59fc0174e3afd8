"""GB300 (sm_103a) Vecchia likelihood library -- Python binding.

A thin ctypes layer over the C ABI in ``include/vecchia.h`` (library
``libvecchia_gb300.so``, built by ``builder.py``).  It only marshals arguments: every
step of the likelihood pass runs in the library's CUDA kernels.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library is missing, every
call raises.

Entry points (same names as the C ABI):
  * ``vecchia_loglik_grad_info``       -- device-resident pass, asynchronous on a stream
  * ``vecchia_loglik_grad_info_host``  -- end-to-end pass from host (numpy) arrays
  * ``vecchia_covariance_pairs``       -- the device covariance functions on explicit pairs
  * ``vecchia_fit``                    -- Fisher scoring on the device (CUDA graph)
  * ``vecchia_batch_loglik_grad_info`` -- the pass for many datasets in one launch
  * ``vecchia_batch_fit``              -- Fisher scoring for many datasets at once
  * ``vecchia_autotune`` / ``vecchia_batch_autotune`` -- kernel-mapping autotuner
  * ``vecchia_fields_*``               -- many fields at shared locations: pass, fit,
                                          simulation, semivariogram features, learned start
  * ``vecchia_mlp_*``                  -- the learned start's network (forward, gradient,
                                          Adam step); training pipeline in ``warmstart``
Covariance functions (parameter order): EXP_ISO (sigma2, rho, tau2), MATERN_ISO (sigma2,
rho, nu, tau2), EXP_SPACETIME (sigma2, rho_s, rho_t, tau2); nugget = sigma2 * tau2.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvecchia_gb300.so")

EXP_ISO, MATERN_ISO, EXP_SPACETIME, EXP_ANISO = 0, 1, 2, 3
FP64, MIXED = 0, 1
NPARMS = {EXP_ISO: 3, MATERN_ISO: 4, EXP_SPACETIME: 4}   # EXP_ANISO: d + 2, see nparms()
STATUS = {0: "VEC_OK", 1: "VEC_ERR_ARG", 2: "VEC_ERR_NOT_PD", 3: "VEC_ERR_NONFINITE",
          4: "VEC_ERR_NOMEM", 5: "VEC_ERR_CUDA", 6: "VEC_ERR_TIMEOUT", 7: "VEC_ERR_UNSUPPORTED"}
_PREC = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}
FIT_MIXED_ONLY = 2   # vecchia_fit only: mixed-precision passes throughout


class FitOpts(ctypes.Structure):
    """vec_fit_opts (include/vecchia.h)."""
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("max_halvings", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("prec", ctypes.c_int)]


class FitInfo(ctypes.Structure):
    """vec_fit_info (include/vecchia.h)."""
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("evals", ctypes.c_int),
                ("pass_status", ctypes.c_int)]


FIT_STATUS = {0: "converged", 1: "iteration limit", 2: "no ascent step", 3: "start failed"}


class VecchiaError(RuntimeError):
    def __init__(self, code: int, msg: str, bad_index: int = -1):
        super().__init__("%s: %s" % (STATUS.get(code, "?"), msg))
        self.code = code
        self.bad_index = bad_index


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compiles the CUDA library in-tree (nvcc, sm_103a) and returns its path."""
    from . import builder
    return builder.build(force=force)


def lib():
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("the CUDA library %s is not built; run "
                               "paper_2407_02740_gb300.build() (no CPU fallback exists)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.vecchia_create.argtypes = [ctypes.POINTER(P), ci]
        L.vecchia_destroy.argtypes = [P]
        L.vecchia_last_error.restype = ctypes.c_char_p
        L.vecchia_nparms.argtypes = [ci]
        L.vecchia_nparms_d.argtypes = [ci, ci]
        L.vecchia_measure_peaks.argtypes = [P, P]
        L.vecchia_group_blocks.argtypes = [P, i64, ci, P, i64, P, P, P, P]
        L.vecchia_group_classes.argtypes = [P, i64, ci, P, P, P]
        L.vecchia_grouped_loglik_grad_info.argtypes = [P, P, P, P, i64, ci, ci, i64, P, P, P, P,
                                                       ci, P, P, P, ci, ci, P, P, P]
        L.vecchia_set_lanes.argtypes = [P, ci]
        L.vecchia_set_block_threads.argtypes = [P, ci]
        L.vecchia_set_group_chunk.argtypes = [P, ci]
        L.vecchia_set_matern_table.argtypes = [P, ci]
        L.vecchia_autotune.argtypes = [P, P, P, P, P, i64, ci, ci, ci, P, ci, ci, P, ci, P, P, P]
        L.vecchia_autotune_save.argtypes = [P, ctypes.c_char_p]
        L.vecchia_autotune_load.argtypes = [P, ctypes.c_char_p]
        L.vecchia_set_timing.argtypes = [P, ci]
        L.vecchia_last_timing.argtypes = [P, P, P, P]
        L.vecchia_kernels_per_pass.argtypes = [ci]
        L.vecchia_loglik_grad_info.argtypes = [P, P, P, P, P, i64, ci, ci, ci, P, ci, ci, P, P, P]
        L.vecchia_loglik_grad_info_host.argtypes = [P, P, P, P, P, i64, ci, ci, ci, P, ci, ci,
                                                    P, P, P, P, P]
        L.vecchia_covariance_pairs.argtypes = [P, ci, P, ci, i64, P, P, P, P, P, P]
        L.vecchia_batch_loglik_grad_info.argtypes = [P, ci, P, P, P, P, P, P, ci, ci, P, ci, ci,
                                                     P, P, P]
        L.vecchia_fit.argtypes = [P, P, P, P, P, i64, ci, ci, ci, ci, P, ctypes.POINTER(FitOpts),
                                  P, P, P, P, P, P, ctypes.POINTER(FitInfo)]
        L.vecchia_loglik_grad_info_noalloc.argtypes = [P, P, P, P, i64, ci, ci, ci, P, ci, ci,
                                                       P, P, P]
        L.vecchia_batch_fit.argtypes = [P, ci, P, P, P, P, P, P, ci, ci, ci, P,
                                        ctypes.POINTER(FitOpts), P, P, P, P]
        L.vecchia_batch_autotune.argtypes = [P, ci, P, P, P, P, P, P, ci, ci, P, ci, ci, P, ci,
                                             P, P, P]
        L.vecchia_batch_plan_create.argtypes = [P, ci, P, P, ci, ci, ci, ci, ctypes.POINTER(P)]
        L.vecchia_batch_plan_run.argtypes = [P, P, P, P, P, P, P, P, P]
        L.vecchia_batch_plan_mapping.argtypes = [P, P, P, P]
        L.vecchia_batch_plan_class.argtypes = [P, ci, P, P, P, P]
        L.vecchia_batch_plan_destroy.argtypes = [P]
        L.vecchia_fields_loglik_grad_info.argtypes = [P, ci, P, P, P, i64, ci, ci, ci, P, P, ci,
                                                      ci, P, P, P]
        L.vecchia_fields_fit.argtypes = [P, ci, P, P, P, i64, ci, ci, ci, P, ci, P,
                                         ctypes.POINTER(FitOpts), P, P, P, P]
        L.vecchia_fields_simulate.argtypes = [P, ci, P, P, i64, ci, ci, P, ci, P, P, P, P]
        L.vecchia_fields_variogram.argtypes = [P, ci, P, P, i64, ci, ci, P, P, i64, P, ci, P, P, P,
                                               P]
        cf = ctypes.c_float
        L.vecchia_ordered_nn.argtypes = [P, P, i64, ci, ci, P, P]
        L.vecchia_nearest.argtypes = [P, P, i64, P, i64, ci, ci, P, P]
        L.vecchia_predict.argtypes = [P, P, P, P, i64, P, P, P, P, i64, ci, ci, ci, P, ci, ci, P,
                                      P, P, P]
        L.vecchia_mlp_forward.argtypes = [P, P, P, P, ci, P, P]
        L.vecchia_mlp_grad.argtypes = [P, P, P, P, P, P, ci, P, P, P]
        L.vecchia_mlp_adam_step.argtypes = [P, P, P, P, ci, cf, P, P, P, P, ci, P, P]
        L.vecchia_mlp_column_moments.argtypes = [P, P, ci, ci, P, P, P]
        L.vecchia_fields_moments.argtypes = [P, ci, i64, P, P, P, P]
        L.vecchia_maxmin_order.argtypes = [P, P, i64, ci, P, P]
        L.vecchia_mlp_targets.argtypes = [P, ci, P, P, P, P, P, P]
        L.vecchia_mlp_theta.argtypes = [P, ci, P, P, P, P]
        L.vecchia_fields_warm_start.argtypes = [P, P, P, ci, P, P, P, i64, ci, ci, ci, P, P, i64,
                                                P, P, ci, P, P, P, P]
        for f in (L.vecchia_create, L.vecchia_destroy, L.vecchia_set_lanes, L.vecchia_set_block_threads,
                  L.vecchia_set_group_chunk, L.vecchia_set_matern_table,
                  L.vecchia_loglik_grad_info, L.vecchia_loglik_grad_info_host,
                  L.vecchia_covariance_pairs, L.vecchia_nparms, L.vecchia_nparms_d, L.vecchia_max_m,
                  L.vecchia_set_timing, L.vecchia_last_timing, L.vecchia_kernels_per_pass,
                  L.vecchia_loglik_grad_info_noalloc, L.vecchia_fit, L.vecchia_autotune,
                  L.vecchia_autotune_save, L.vecchia_autotune_load,
                  L.vecchia_batch_loglik_grad_info, L.vecchia_batch_fit,
                  L.vecchia_batch_autotune, L.vecchia_batch_plan_create,
                  L.vecchia_batch_plan_run, L.vecchia_batch_plan_mapping,
                  L.vecchia_batch_plan_class,
                  L.vecchia_batch_plan_destroy, L.vecchia_fields_loglik_grad_info,
                  L.vecchia_fields_fit, L.vecchia_fields_simulate,
                  L.vecchia_fields_variogram, L.vecchia_mlp_forward, L.vecchia_mlp_grad,
                  L.vecchia_mlp_adam_step, L.vecchia_mlp_column_moments,
                  L.vecchia_fields_moments, L.vecchia_mlp_targets, L.vecchia_mlp_theta,
                  L.vecchia_maxmin_order,
                  L.vecchia_fields_warm_start, L.vecchia_ordered_nn, L.vecchia_nearest,
                  L.vecchia_predict, L.vecchia_measure_peaks, L.vecchia_group_blocks,
                  L.vecchia_group_classes, L.vecchia_grouped_loglik_grad_info):
            f.restype = ci
        _lib = L
    return _lib


def nparms(covfun: int, d: int) -> int:
    """Number of covariance parameters of a family on d-dimensional locations (the
    library's vecchia_nparms_d); raises ValueError if the family does not take d."""
    q = lib().vecchia_nparms_d(int(covfun), int(d))
    if q < 0:
        raise ValueError("covariance function %d does not take d = %d" % (covfun, d))
    return q


def _check(code: int, bad_index: int = -1):
    if code != 0:
        raise VecchiaError(code, lib().vecchia_last_error().decode(), bad_index)


class Handle:
    """Owns a vec_handle (device scratch + stream) on one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().vecchia_create(ctypes.byref(self._h), device))
        self.device = device

    @property
    def ptr(self):
        return self._h

    def set_lanes(self, lanes: int):
        _check(lib().vecchia_set_lanes(self._h, lanes))

    def set_block_threads(self, threads: int):
        _check(lib().vecchia_set_block_threads(self._h, threads))

    def set_group_chunk(self, chunk: int):
        """Grouped pass: members whose terms are formed together (0 = library's choice)."""
        _check(lib().vecchia_set_group_chunk(self._h, chunk))

    def set_matern_table(self, placement):
        """"shared", "global" or "auto" (see vecchia_set_matern_table)."""
        code = {"shared": 1, "global": 0, "auto": -1}.get(placement, placement)
        _check(lib().vecchia_set_matern_table(self._h, int(code)))

    def set_timing(self, enable: bool = True):
        _check(lib().vecchia_set_timing(self._h, 1 if enable else 0))

    def last_timing(self) -> dict:
        """Durations (ms) of the last traced pass: setup, pass kernel, profile kernel."""
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        _check(lib().vecchia_last_timing(self._h, ctypes.byref(a), ctypes.byref(b),
                                         ctypes.byref(c)))
        return {"setup": a.value, "pass": b.value, "profile": c.value}

    def autotune_save(self, path: str):
        _check(lib().vecchia_autotune_save(self._h, path.encode()))

    def autotune_load(self, path: str):
        _check(lib().vecchia_autotune_load(self._h, path.encode()))

    def close(self):
        if self._h:
            lib().vecchia_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles: dict = {}


def default_handle(device: int = 0) -> Handle:
    h = _handles.get(device)
    if h is None:
        h = _handles[device] = Handle(device)
    return h


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _dev_tensor_check(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be contiguous %s" % (name, dtype))


def vecchia_loglik_grad_info(locs, y, X, NNarray, covparms, covfun: int, prec="fp64",
                             stream=None, out=None, status=None, handle: Handle | None = None):
    """Device-resident pass (asynchronous).  Tensors must be CUDA, contiguous: locs (n, d)
    float64, y (n,) float64, X (n, p) float64, NNarray (n, m+1) int32, covparms (q,) float64.
    Returns (out, status): out = [loglik, grad(q), info(q*q), betahat(p)] float64 and
    status = [code, first failing observation] int64, both on the device."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                      (X, torch.float64, "X"), (NNarray, torch.int32, "NNarray"),
                      (covparms, torch.float64, "covparms")):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    p = X.shape[1]
    m = NNarray.shape[1] - 1
    q = nparms(covfun, d)
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if out is None:
        out = torch.empty(1 + q + q * q + p, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(2, dtype=torch.int64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    sptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().vecchia_loglik_grad_info(handle.ptr, _dptr(locs), _dptr(y), _dptr(X),
                                          _dptr(NNarray), n, d, p, m, _dptr(covparms), covfun,
                                          _PREC[prec], sptr, _dptr(out), _dptr(status)))
    return out, status


def vecchia_batch_loglik_grad_info(locs, y, X, NNarray, point_offsets, m, covparms, covfun: int,
                                   prec="fp64", stream=None, out=None, status=None,
                                   handle: Handle | None = None):
    """Batched pass over concatenated datasets (see include/vecchia.h).  locs, y, X,
    NNarray (flat int32, per-dataset NNarrays with local indices, concatenated) and covparms
    (nbatch x q) are CUDA tensors; point_offsets (nbatch+1) and m (nbatch) are host
    sequences.  Returns (out (nbatch, 1+q+q*q+p), status (nbatch, 2)) on the device."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                      (X, torch.float64, "X"), (NNarray, torch.int32, "NNarray"),
                      (covparms, torch.float64, "covparms")):
        _dev_tensor_check(t, dt, nm)
    off = np.ascontiguousarray(point_offsets, dtype=np.int64)
    mm = np.ascontiguousarray(m, dtype=np.int32)
    nb = len(mm)
    d = locs.shape[1]
    p = X.shape[1]
    q = nparms(covfun, d)
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if out is None:
        out = torch.empty(nb, 1 + q + q * q + p, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(nb, 2, dtype=torch.int64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().vecchia_batch_loglik_grad_info(handle.ptr, nb, _dptr(locs), _dptr(y), _dptr(X),
                                                _dptr(NNarray), P(off), P(mm), d, p,
                                                _dptr(covparms), covfun, _PREC[prec],
                                                ctypes.c_void_p(stream.cuda_stream), _dptr(out),
                                                _dptr(status)))
    return out, status


def _batch_common(locs, y, X, NNarray, point_offsets, m, extra=()):
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                      (X, torch.float64, "X"), (NNarray, torch.int32, "NNarray")) + tuple(extra):
        _dev_tensor_check(t, dt, nm)
    off = np.ascontiguousarray(point_offsets, dtype=np.int64)
    mm = np.ascontiguousarray(m, dtype=np.int32)
    if off.shape != (len(mm) + 1,):
        raise ValueError("point_offsets needs nbatch + 1 entries")
    return off, mm


class BatchPlan:
    """vec_batch_plan (include/vecchia.h): the batch description prepared once; ``run``
    only launches kernels and may be captured into a CUDA graph (torch.cuda.graph)."""

    def __init__(self, point_offsets, m, d: int, p: int, covfun: int, prec="fp64",
                 handle: Handle | None = None, device: int = 0):
        self._p = ctypes.c_void_p()
        off = np.ascontiguousarray(point_offsets, dtype=np.int64)
        mm = np.ascontiguousarray(m, dtype=np.int32)
        if off.shape != (len(mm) + 1,):
            raise ValueError("point_offsets needs nbatch + 1 entries")
        if handle is None:
            handle = default_handle(device)
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(lib().vecchia_batch_plan_create(handle.ptr, len(mm), P(off), P(mm), d, p, covfun,
                                               _PREC[prec], ctypes.byref(self._p)))
        self.nbatch, self.d, self.p, self.covfun = len(mm), d, p, covfun

    def mapping(self) -> dict:
        """Lanes and threads of the class with the most observations, all tiles, and per
        class of datasets (by block size) its largest m, mapping and tiles."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().vecchia_batch_plan_mapping(self._p, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c)))
        classes = []
        for k in range(3):
            mm, la, th, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            _check(lib().vecchia_batch_plan_class(self._p, k, ctypes.byref(mm), ctypes.byref(la),
                                                  ctypes.byref(th), ctypes.byref(nt)))
            if mm.value >= 0:
                classes.append({"mmax": mm.value, "lanes": la.value, "threads": th.value,
                                "ntiles": nt.value})
        return {"lanes": a.value, "threads": b.value, "ntiles": c.value, "classes": classes}

    def run(self, locs, y, X, NNarray, covparms, out, status, stream=None):
        """Enqueues the batched pass; out (nbatch, 1+q+q*q+p) and status (nbatch, 2) are
        caller-provided CUDA tensors."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(locs.device)
        _check(lib().vecchia_batch_plan_run(self._p, _dptr(locs), _dptr(y), _dptr(X),
                                            _dptr(NNarray), _dptr(covparms),
                                            ctypes.c_void_p(stream.cuda_stream), _dptr(out),
                                            _dptr(status)))

    def close(self):
        if self._p:
            lib().vecchia_batch_plan_destroy(self._p)
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vecchia_batch_fit(locs, y, X, NNarray, point_offsets, m, covfun: int, start,
                      tol: float = 1e-4, maxit: int = 40, max_halvings: int = 10,
                      use_graph: bool = True, prec="fp64", stream=None,
                      handle: Handle | None = None) -> dict:
    """Fisher scoring for many datasets at once (see vecchia_batch_fit in
    include/vecchia.h).  Data as for vecchia_batch_loglik_grad_info; start is a CUDA
    tensor (nbatch, q).  Returns theta (nbatch, q) and out (nbatch, 1+q+q*q+p) as CUDA
    tensors and status / iters / evals / pass_status as numpy arrays."""
    import torch
    off, mm = _batch_common(locs, y, X, NNarray, point_offsets, m,
                            ((start, torch.float64, "start"),))
    nb = len(mm)
    d = locs.shape[1]
    p = X.shape[1]
    q = nparms(covfun, d)
    dev = locs.device
    if tuple(start.shape) != (nb, q):
        raise ValueError("start must be (nbatch, q)")
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    theta = torch.empty(nb, q, dtype=torch.float64, device=dev)
    out = torch.empty(nb, 1 + q + q * q + p, dtype=torch.float64, device=dev)
    infos = (FitInfo * nb)()
    opts = FitOpts(tol, maxit, max_halvings, 1 if use_graph else 0,
                   FIT_MIXED_ONLY if prec == "mixed_only" else _PREC[prec])
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().vecchia_batch_fit(handle.ptr, nb, _dptr(locs), _dptr(y), _dptr(X), _dptr(NNarray),
                                   P(off), P(mm), d, p, covfun, _dptr(start), ctypes.byref(opts),
                                   ctypes.c_void_p(stream.cuda_stream), _dptr(theta), _dptr(out),
                                   ctypes.cast(infos, ctypes.c_void_p)))
    return {"theta": theta, "out": out,
            "status": np.array([f.status for f in infos]),
            "iters": np.array([f.iters for f in infos]),
            "evals": np.array([f.evals for f in infos]),
            "pass_status": np.array([f.pass_status for f in infos])}


def vecchia_batch_autotune(locs, y, X, NNarray, point_offsets, m, covparms, covfun: int,
                           prec="fp64", reps: int = 3, stream=None,
                           handle: Handle | None = None) -> dict:
    """Times every kernel mapping of the batched pass on these inputs and records the
    fastest in the handle (see vecchia_batch_autotune in include/vecchia.h)."""
    import torch
    off, mm = _batch_common(locs, y, X, NNarray, point_offsets, m,
                            ((covparms, torch.float64, "covparms"),))
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    lanes, threads, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().vecchia_batch_autotune(handle.ptr, len(mm), _dptr(locs), _dptr(y), _dptr(X),
                                        _dptr(NNarray), P(off), P(mm), locs.shape[1], X.shape[1],
                                        _dptr(covparms), covfun, _PREC[prec],
                                        ctypes.c_void_p(stream.cuda_stream), reps,
                                        ctypes.byref(lanes), ctypes.byref(threads),
                                        ctypes.byref(ms)))
    return {"lanes": lanes.value, "threads": threads.value, "ms": ms.value}


def _fields_common(locs, X, NNarray, Y, extra=()):
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (X, torch.float64, "X"),
                      (NNarray, torch.int32, "NNarray"), (Y, torch.float64, "Y")) + tuple(extra):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    if NNarray.shape[0] != n or X.shape[0] != n or Y.dim() != 2 or Y.shape[1] != n:
        raise ValueError("shapes: locs (n, d), X (n, p), NNarray (n, m+1), Y (nfields, n)")
    return n, d, X.shape[1], NNarray.shape[1] - 1, Y.shape[0]


def vecchia_fields_loglik_grad_info(locs, X, NNarray, Y, covparms, covfun: int, prec="fp64",
                                    stream=None, out=None, status=None,
                                    handle: Handle | None = None):
    """The pass for nfields fields at shared locations (see include/vecchia.h).  Y is
    (nfields, n), covparms (nfields, q).  Returns (out, status) on the device."""
    import torch
    n, d, p, m, nf = _fields_common(locs, X, NNarray, Y, ((covparms, torch.float64, "covparms"),))
    q = nparms(covfun, d)
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if out is None:
        out = torch.empty(nf, 1 + q + q * q + p, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(nf, 2, dtype=torch.int64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    _check(lib().vecchia_fields_loglik_grad_info(handle.ptr, nf, _dptr(locs), _dptr(X),
                                                 _dptr(NNarray), n, d, p, m, _dptr(Y),
                                                 _dptr(covparms), covfun, _PREC[prec],
                                                 ctypes.c_void_p(stream.cuda_stream), _dptr(out),
                                                 _dptr(status)))
    return out, status


def vecchia_fields_fit(locs, X, NNarray, Y, covfun: int, start, tol: float = 1e-4,
                       maxit: int = 40, max_halvings: int = 10, use_graph: bool = True,
                       prec="fp64", stream=None, handle: Handle | None = None) -> dict:
    """Fisher scoring for nfields fields at shared locations (see vecchia_fields_fit);
    start is a CUDA tensor (nfields, q).  Same result dictionary as vecchia_batch_fit."""
    import torch
    n, d, p, m, nf = _fields_common(locs, X, NNarray, Y, ((start, torch.float64, "start"),))
    q = nparms(covfun, d)
    dev = locs.device
    if tuple(start.shape) != (nf, q):
        raise ValueError("start must be (nfields, q)")
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    theta = torch.empty(nf, q, dtype=torch.float64, device=dev)
    out = torch.empty(nf, 1 + q + q * q + p, dtype=torch.float64, device=dev)
    infos = (FitInfo * nf)()
    opts = FitOpts(tol, maxit, max_halvings, 1 if use_graph else 0,
                   FIT_MIXED_ONLY if prec == "mixed_only" else _PREC[prec])
    _check(lib().vecchia_fields_fit(handle.ptr, nf, _dptr(locs), _dptr(X), _dptr(NNarray), n, d,
                                    p, m, _dptr(Y), covfun, _dptr(start), ctypes.byref(opts),
                                    ctypes.c_void_p(stream.cuda_stream), _dptr(theta), _dptr(out),
                                    ctypes.cast(infos, ctypes.c_void_p)))
    return {"theta": theta, "out": out,
            "status": np.array([f.status for f in infos]),
            "iters": np.array([f.iters for f in infos]),
            "evals": np.array([f.evals for f in infos]),
            "pass_status": np.array([f.pass_status for f in infos])}


def vecchia_fields_simulate(locs, NNarray, covparms, covfun: int, z, stream=None,
                            handle: Handle | None = None):
    """Sequential Vecchia draws (see vecchia_fields_simulate): z (nfields, n) standard
    normal variates on the device, covparms (nfields, q).  Returns (y, status)."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (NNarray, torch.int32, "NNarray"),
                      (covparms, torch.float64, "covparms"), (z, torch.float64, "z")):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    m = NNarray.shape[1] - 1
    nf = z.shape[0]
    if z.dim() != 2 or z.shape[1] != n or NNarray.shape[0] != n:
        raise ValueError("shapes: locs (n, d), NNarray (n, m+1), z (nfields, n)")
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    y = torch.empty_like(z)
    status = torch.empty(nf, 2, dtype=torch.int64, device=dev)
    _check(lib().vecchia_fields_simulate(handle.ptr, nf, _dptr(locs), _dptr(NNarray), n, d, m,
                                         _dptr(covparms), covfun, _dptr(z),
                                         ctypes.c_void_p(stream.cuda_stream), _dptr(y),
                                         _dptr(status)))
    return y, status


def vecchia_fields_variogram(locs, NNarray, Y, rand_pairs, edges2, stream=None, raw=False,
                             handle: Handle | None = None):
    """Binned semivariogram features (see vecchia_fields_variogram): Y (nfields, n),
    rand_pairs (npairs, 2) uint32 as an int32 CUDA tensor (same bits), edges2 (nbins+1)
    squared lag edges.  Returns features (nfields, nbins) float32, and with raw=True also
    the bin sums and counts."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (NNarray, torch.int32, "NNarray"),
                      (Y, torch.float64, "Y"), (edges2, torch.float64, "edges2"),
                      (rand_pairs, torch.int32, "rand_pairs")):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    m = NNarray.shape[1] - 1
    nf = Y.shape[0]
    nb = edges2.shape[0] - 1
    npairs = rand_pairs.shape[0]
    if Y.dim() != 2 or Y.shape[1] != n or (npairs and rand_pairs.shape[1] != 2):
        raise ValueError("shapes: locs (n, d), Y (nfields, n), rand_pairs (npairs, 2)")
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    feats = torch.empty(nf, nb, dtype=torch.float32, device=dev)
    bs = torch.empty(nf, nb, dtype=torch.float64, device=dev) if raw else None
    bc = torch.empty(nf, nb, dtype=torch.int64, device=dev) if raw else None
    _check(lib().vecchia_fields_variogram(handle.ptr, nf, _dptr(locs), _dptr(NNarray), n, d, m,
                                          _dptr(Y), _dptr(rand_pairs) if npairs else None, npairs,
                                          _dptr(edges2), nb, ctypes.c_void_p(stream.cuda_stream),
                                          _dptr(feats), _dptr(bs) if raw else None,
                                          _dptr(bc) if raw else None))
    return (feats, bs, bc) if raw else feats


def vecchia_ordered_nn(locs, m: int, stream=None, handle: Handle | None = None):
    """NNarray (n, m+1) int32 on the device for locations already in their ordering (see
    vecchia_ordered_nn in include/vecchia.h)."""
    import torch
    _dev_tensor_check(locs, torch.float64, "locs")
    n, d = locs.shape
    handle = handle or default_handle(locs.device.index or 0)
    NN = torch.empty(n, m + 1, dtype=torch.int32, device=locs.device)
    _check(lib().vecchia_ordered_nn(handle.ptr, _dptr(locs), n, d, m,
                                    ctypes.c_void_p(_stream(locs, stream).cuda_stream), _dptr(NN)))
    return NN


def vecchia_nearest(locs_ref, locs_query, m: int, stream=None, handle: Handle | None = None):
    """(nquery, m) int32 indices of the m nearest reference locations of each query."""
    import torch
    _dev_tensor_check(locs_ref, torch.float64, "locs_ref")
    _dev_tensor_check(locs_query, torch.float64, "locs_query")
    handle = handle or default_handle(locs_ref.device.index or 0)
    NN = torch.empty(locs_query.shape[0], m, dtype=torch.int32, device=locs_ref.device)
    _check(lib().vecchia_nearest(handle.ptr, _dptr(locs_ref), locs_ref.shape[0], _dptr(locs_query),
                                 locs_query.shape[0], locs_ref.shape[1], m,
                                 ctypes.c_void_p(_stream(locs_ref, stream).cuda_stream), _dptr(NN)))
    return NN


def vecchia_predict(locs, y, X, beta, locs_pred, X_pred, NN_pred, covparms, covfun: int,
                    latent: bool = True, stream=None, handle: Handle | None = None):
    """Vecchia prediction (see vecchia_predict in include/vecchia.h).  Returns (mean, var,
    status) as CUDA tensors."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                      (X, torch.float64, "X"), (beta, torch.float64, "beta"),
                      (locs_pred, torch.float64, "locs_pred"), (X_pred, torch.float64, "X_pred"),
                      (NN_pred, torch.int32, "NN_pred"), (covparms, torch.float64, "covparms")):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    npred, m = NN_pred.shape
    handle = handle or default_handle(locs.device.index or 0)
    mean = torch.empty(npred, dtype=torch.float64, device=locs.device)
    var = torch.empty_like(mean)
    status = torch.empty(2, dtype=torch.int64, device=locs.device)
    _check(lib().vecchia_predict(handle.ptr, _dptr(locs), _dptr(y), _dptr(X), n, _dptr(beta),
                                 _dptr(locs_pred), _dptr(X_pred), _dptr(NN_pred), npred, d,
                                 X.shape[1], m, _dptr(covparms), covfun, 1 if latent else 0,
                                 ctypes.c_void_p(_stream(locs, stream).cuda_stream), _dptr(mean),
                                 _dptr(var), _dptr(status)))
    return mean, var, status


MLP_NPARAMS, MLP_NNORM = 21252, 72


def _stream(t, stream):
    import torch
    return torch.cuda.current_stream(t.device) if stream is None else stream


def vecchia_mlp_forward(params, norm, X, stream=None, handle: Handle | None = None):
    """Predictions (nsamples, 4) of the learned-start network (see include/vecchia.h)."""
    import torch
    for t, nm in ((params, "params"), (norm, "norm"), (X, "X")):
        _dev_tensor_check(t, torch.float32, nm)
    handle = handle or default_handle(X.device.index or 0)
    out = torch.empty(X.shape[0], 4, dtype=torch.float32, device=X.device)
    _check(lib().vecchia_mlp_forward(handle.ptr, _dptr(params), _dptr(norm), _dptr(X), X.shape[0],
                                     ctypes.c_void_p(_stream(X, stream).cuda_stream), _dptr(out)))
    return out


def _index_arg(index, X):
    import torch
    if index is None:
        return None, X.shape[0]
    _dev_tensor_check(index, torch.int32, "index")
    return _dptr(index), index.shape[0]


def vecchia_mlp_grad(params, norm, X, T, index=None, stream=None, handle: Handle | None = None):
    """(gradient, loss) of the mean squared error on standardised targets over the rows
    `index` (int32 CUDA tensor) of X and T, or all rows."""
    import torch
    for t, nm in ((params, "params"), (norm, "norm"), (X, "X"), (T, "T")):
        _dev_tensor_check(t, torch.float32, nm)
    handle = handle or default_handle(X.device.index or 0)
    ip, ns = _index_arg(index, X)
    g = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(lib().vecchia_mlp_grad(handle.ptr, _dptr(params), _dptr(norm), _dptr(X), _dptr(T), ip,
                                  ns, ctypes.c_void_p(_stream(X, stream).cuda_stream), _dptr(g),
                                  _dptr(loss)))
    return g, loss


def vecchia_mlp_adam_step(params, adam_m, adam_v, step: int, lr: float, norm, X, T, index=None,
                          loss=None, stream=None, handle: Handle | None = None):
    """One Adam step in place on params (moment buffers adam_m, adam_v) over the rows
    `index` of X and T (a minibatch), or all rows."""
    import torch
    for t, nm in ((params, "params"), (adam_m, "adam_m"), (adam_v, "adam_v"), (norm, "norm"),
                  (X, "X"), (T, "T")):
        _dev_tensor_check(t, torch.float32, nm)
    handle = handle or default_handle(X.device.index or 0)
    ip, ns = _index_arg(index, X)
    _check(lib().vecchia_mlp_adam_step(handle.ptr, _dptr(params), _dptr(adam_m), _dptr(adam_v),
                                       int(step), float(lr), _dptr(norm), _dptr(X), _dptr(T), ip,
                                       ns, ctypes.c_void_p(_stream(X, stream).cuda_stream),
                                       _dptr(loss) if loss is not None else None))


def vecchia_mlp_column_moments(X, stream=None, handle: Handle | None = None):
    """Column means and standard deviations of a float32 CUDA matrix."""
    import torch
    _dev_tensor_check(X, torch.float32, "X")
    handle = handle or default_handle(X.device.index or 0)
    mean = torch.empty(X.shape[1], dtype=torch.float32, device=X.device)
    sd = torch.empty_like(mean)
    _check(lib().vecchia_mlp_column_moments(handle.ptr, _dptr(X), X.shape[0], X.shape[1],
                                            ctypes.c_void_p(_stream(X, stream).cuda_stream),
                                            _dptr(mean), _dptr(sd)))
    return mean, sd


def vecchia_maxmin_order(locs, stream=None, handle: Handle | None = None):
    """Maxmin ordering of the rows of a float64 CUDA tensor locs (n, d), d <= 3, on the
    device: returns the int64 CUDA tensor of original indices in maxmin order."""
    import torch
    _dev_tensor_check(locs, torch.float64, "locs")
    n, d = locs.shape
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    order = torch.empty(n, dtype=torch.int64, device=dev)
    _check(lib().vecchia_maxmin_order(handle.ptr, _dptr(locs), n, d,
                                      ctypes.c_void_p(stream.cuda_stream), _dptr(order)))
    return order


def vecchia_fields_moments(Y, stream=None, handle: Handle | None = None):
    """Mean and population variance (float64) of each row of a float64 CUDA matrix Y
    (nfields, n)."""
    import torch
    _dev_tensor_check(Y, torch.float64, "Y")
    if Y.dim() != 2:
        raise ValueError("Y must be (nfields, n)")
    handle = handle or default_handle(Y.device.index or 0)
    mean = torch.empty(Y.shape[0], dtype=torch.float64, device=Y.device)
    var = torch.empty_like(mean)
    _check(lib().vecchia_fields_moments(handle.ptr, Y.shape[0], Y.shape[1], _dptr(Y),
                                        ctypes.c_void_p(_stream(Y, stream).cuda_stream),
                                        _dptr(mean), _dptr(var)))
    return mean, var


def vecchia_mlp_targets(theta, var, lo, hi, stream=None, handle: Handle | None = None):
    """Training targets (nfields, 4) float32 from fitted MATERN_ISO parameters theta
    (nfields, 4) float64 and the fields' variances var (nfields): (log(sigma2 / var),
    log rho, log nu, log tau2), component j clamped to [log lo[j], log hi[j]]."""
    import torch
    _dev_tensor_check(theta, torch.float64, "theta")
    _dev_tensor_check(var, torch.float64, "var")
    nf = theta.shape[0]
    if theta.dim() != 2 or theta.shape[1] != 4 or var.shape[0] != nf:
        raise ValueError("theta (nfields, 4), var (nfields)")
    handle = handle or default_handle(theta.device.index or 0)
    T = torch.empty(nf, 4, dtype=torch.float32, device=theta.device)
    lo_ = (ctypes.c_double * 4)(*[float(v) for v in lo])
    hi_ = (ctypes.c_double * 4)(*[float(v) for v in hi])
    _check(lib().vecchia_mlp_targets(handle.ptr, nf, _dptr(theta), _dptr(var), lo_, hi_,
                                     ctypes.c_void_p(_stream(theta, stream).cuda_stream),
                                     _dptr(T)))
    return T


def vecchia_mlp_theta(pred, var, stream=None, handle: Handle | None = None):
    """theta0 (nfields, 4) float64 from network outputs pred (nfields, 4) float32 and the
    fields' variances: (var e^t0, e^t1, e^t2 clamped to [0.05, 20], e^t3)."""
    import torch
    _dev_tensor_check(pred, torch.float32, "pred")
    _dev_tensor_check(var, torch.float64, "var")
    nf = pred.shape[0]
    if pred.dim() != 2 or pred.shape[1] != 4 or var.shape[0] != nf:
        raise ValueError("pred (nfields, 4), var (nfields)")
    handle = handle or default_handle(pred.device.index or 0)
    th = torch.empty(nf, 4, dtype=torch.float64, device=pred.device)
    _check(lib().vecchia_mlp_theta(handle.ptr, nf, _dptr(pred), _dptr(var),
                                   ctypes.c_void_p(_stream(pred, stream).cuda_stream), _dptr(th)))
    return th


def vecchia_fields_warm_start(params, norm, locs, X, NNarray, Y, rand_pairs, edges2,
                              default_start, prec="fp64", stream=None,
                              handle: Handle | None = None):
    """Learned starting points with the default-start fallback (see include/vecchia.h).
    Returns (start (nfields, 4) float64, used_learned (nfields) int32, features)."""
    import torch
    n, d, p, m, nf = _fields_common(locs, X, NNarray, Y, ((default_start, torch.float64, "default_start"),
                                                          (edges2, torch.float64, "edges2"),
                                                          (rand_pairs, torch.int32, "rand_pairs")))
    for t, nm in ((params, "params"), (norm, "norm")):
        _dev_tensor_check(t, torch.float32, nm)
    handle = handle or default_handle(locs.device.index or 0)
    start = torch.empty(nf, 4, dtype=torch.float64, device=locs.device)
    used = torch.empty(nf, dtype=torch.int32, device=locs.device)
    feats = torch.empty(nf, 32, dtype=torch.float32, device=locs.device)
    _check(lib().vecchia_fields_warm_start(handle.ptr, _dptr(params), _dptr(norm), nf, _dptr(locs),
                                           _dptr(X), _dptr(NNarray), n, d, p, m, _dptr(Y),
                                           _dptr(rand_pairs), rand_pairs.shape[0], _dptr(edges2),
                                           _dptr(default_start), _PREC[prec],
                                           ctypes.c_void_p(_stream(locs, stream).cuda_stream),
                                           _dptr(start), _dptr(used), _dptr(feats)))
    return start, used, feats


def vecchia_autotune(locs, y, X, NNarray, covparms, covfun: int, prec="fp64", reps: int = 3,
                     stream=None, handle: Handle | None = None) -> dict:
    """Times every kernel mapping on these inputs and records the fastest in the handle
    (see vecchia_autotune in include/vecchia.h).  Returns lanes, threads and ms."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                      (X, torch.float64, "X"), (NNarray, torch.int32, "NNarray"),
                      (covparms, torch.float64, "covparms")):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    p = X.shape[1]
    m = NNarray.shape[1] - 1
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    lanes, threads, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().vecchia_autotune(handle.ptr, _dptr(locs), _dptr(y), _dptr(X), _dptr(NNarray), n,
                                  d, p, m, _dptr(covparms), covfun, _PREC[prec],
                                  ctypes.c_void_p(stream.cuda_stream), reps, ctypes.byref(lanes),
                                  ctypes.byref(threads), ctypes.byref(ms)))
    return {"lanes": lanes.value, "threads": threads.value, "ms": ms.value}


def vecchia_fit(locs, y, X, NNarray, covfun: int, start, tol: float = 1e-4, maxit: int = 40,
                max_halvings: int = 10, use_graph: bool = True, prec="fp64", stream=None,
                handle: Handle | None = None) -> dict:
    """Fisher scoring on the device (see vecchia_fit in include/vecchia.h).  Data tensors
    are CUDA tensors as for vecchia_loglik_grad_info; start is a host sequence of q values.
    prec: "fp64", "mixed" (mixed phase, then an FP64 phase) or "mixed_only" (mixed passes
    throughout).  Returns theta, betahat, loglik, grad, info (numpy) and status / iters /
    evals."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                      (X, torch.float64, "X"), (NNarray, torch.int32, "NNarray")):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    p = X.shape[1]
    m = NNarray.shape[1] - 1
    q = nparms(covfun, d)
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    st = np.ascontiguousarray(start, dtype=np.float64)
    opts = FitOpts(tol, maxit, max_halvings, 1 if use_graph else 0,
                   FIT_MIXED_ONLY if prec == "mixed_only" else _PREC[prec])
    info_ = FitInfo()
    theta = np.empty(q)
    beta = np.empty(p)
    ll = ctypes.c_double()
    grad = np.empty(q)
    info = np.empty((q, q))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().vecchia_fit(handle.ptr, _dptr(locs), _dptr(y), _dptr(X), _dptr(NNarray), n, d,
                             p, m, covfun, P(st), ctypes.byref(opts),
                             ctypes.c_void_p(stream.cuda_stream), P(theta), P(beta),
                             ctypes.byref(ll), P(grad), P(info), ctypes.byref(info_)))
    return {"theta": theta, "betahat": beta, "loglik": ll.value, "grad": grad, "info": info,
            "status": info_.status, "iters": info_.iters, "evals": info_.evals,
            "pass_status": info_.pass_status}


def vecchia_loglik_grad_info_noalloc(locs, y, X, NNarray, covparms, covfun: int,
                                     prec="fp64", stream=None, out=None, status=None):
    """The device-resident FP64 pass without any device allocation by the library: for
    callers that cannot allocate (GPU memory owned by another allocator or held to a fixed
    budget, loops that cannot take an allocation's synchronisation).  It runs on the
    current CUDA device with the library's static scratch; `out` and `status` are still
    supplied by the caller (allocated here only when not given).  Only prec="fp64" is
    accepted.  Calls that overlap on the GPU share that scratch and must be serialised."""
    import torch
    for t, dt, nm in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                      (X, torch.float64, "X"), (NNarray, torch.int32, "NNarray"),
                      (covparms, torch.float64, "covparms")):
        _dev_tensor_check(t, dt, nm)
    n, d = locs.shape
    p = X.shape[1]
    m = NNarray.shape[1] - 1
    q = nparms(covfun, d)
    dev = locs.device
    if out is None:
        out = torch.empty(1 + q + q * q + p, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(2, dtype=torch.int64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        _check(lib().vecchia_loglik_grad_info_noalloc(
            _dptr(locs), _dptr(y), _dptr(X), _dptr(NNarray), n, d, p, m, _dptr(covparms),
            covfun, _PREC[prec], ctypes.c_void_p(stream.cuda_stream), _dptr(out),
            _dptr(status)))
    return out, status


def unpack(out, q: int, p: int) -> dict:
    """Splits a result vector into loglik, grad, info, betahat (numpy)."""
    o = out.detach().cpu().numpy() if hasattr(out, "detach") else np.asarray(out)
    return {"loglik": float(o[0]), "grad": o[1:1 + q].copy(),
            "info": o[1 + q:1 + q + q * q].reshape(q, q).copy(),
            "betahat": o[1 + q + q * q:1 + q + q * q + p].copy()}


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def vecchia_loglik_grad_info_host(locs, y, X, NNarray, covparms, covfun: int, prec="fp64",
                                  handle: Handle | None = None, device: int = 0) -> dict:
    """End-to-end pass from host arrays (copies in, runs, copies out, synchronises)."""
    locs = _host(locs, np.float64)
    if locs.ndim == 1:
        locs = locs[:, None]
    y = _host(y, np.float64)
    X = _host(X, np.float64)
    if X.ndim == 1:
        X = X[:, None]
    NN = _host(NNarray, np.int32)
    cp = _host(covparms, np.float64)
    n, d = locs.shape
    p = X.shape[1]
    m = NN.shape[1] - 1
    q = nparms(covfun, d)
    if handle is None:
        handle = default_handle(device)
    ll = ctypes.c_double()
    grad = np.empty(q)
    info = np.empty((q, q))
    beta = np.empty(p)
    bad = ctypes.c_int64(-1)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    code = lib().vecchia_loglik_grad_info_host(handle.ptr, P(locs), P(y), P(X), P(NN), n, d, p,
                                               m, P(cp), covfun, _PREC[prec], ctypes.byref(ll),
                                               P(grad), P(info), P(beta), ctypes.byref(bad))
    _check(code, bad.value)
    return {"loglik": ll.value, "grad": grad, "info": info, "betahat": beta,
            "bad_index": bad.value}


def vecchia_group_blocks(NNarray, group_off):
    """Block lists for grouped conditioning from a HOST NNarray (n, m+1) and contiguous group
    boundaries (see vecchia_group_blocks in include/vecchia.h).  Returns numpy arrays
    (block_off int64, block_idx int32, nmemb int32) and kmax."""
    NN = np.ascontiguousarray(NNarray, dtype=np.int32)
    goff = np.ascontiguousarray(group_off, dtype=np.int64)
    n, W = NN.shape
    ng = len(goff) - 1
    off = np.empty(ng + 1, dtype=np.int64)
    kmax = ctypes.c_int()
    P = ctypes.c_void_p
    _check(lib().vecchia_group_blocks(NN.ctypes.data_as(P), n, W - 1, goff.ctypes.data_as(P), ng,
                                      off.ctypes.data_as(P), None, None, ctypes.byref(kmax)))
    idx = np.empty(int(off[-1]), dtype=np.int32)
    nm = np.empty(ng, dtype=np.int32)
    _check(lib().vecchia_group_blocks(NN.ctypes.data_as(P), n, W - 1, goff.ctypes.data_as(P), ng,
                                      off.ctypes.data_as(P), idx.ctypes.data_as(P),
                                      nm.ctypes.data_as(P), ctypes.byref(kmax)))
    return off, idx, nm, kmax.value


def vecchia_group_classes(block_off, nclass: int = 3):
    """Launch classes of the groups by block size (see vecchia_group_classes in
    include/vecchia.h).  Returns numpy (gorder int32, class_off int64, class_kmax int32)."""
    off = np.ascontiguousarray(block_off, dtype=np.int64)
    ng = len(off) - 1
    gorder = np.empty(ng, dtype=np.int32)
    class_off = np.empty(nclass + 1, dtype=np.int64)
    class_kmax = np.empty(nclass, dtype=np.int32)
    P = ctypes.c_void_p
    _check(lib().vecchia_group_classes(off.ctypes.data_as(P), ng, nclass, gorder.ctypes.data_as(P),
                                       class_off.ctypes.data_as(P), class_kmax.ctypes.data_as(P)))
    return gorder, class_off, class_kmax


def vecchia_grouped_loglik_grad_info(locs, y, X, block_off, block_idx, nmemb, kmax, covparms,
                                     covfun: int, prec="fp64", stream=None, out=None,
                                     status=None, handle: Handle | None = None, classes=None):
    """Grouped-conditioning pass (see include/vecchia.h).  CUDA tensors: locs (n, d), y (n,),
    X (n, p) float64, block_off int64, block_idx int32, nmemb int32, covparms float64.  kmax
    is the largest block (one launch), unless classes = (gorder CUDA int32, class_off,
    class_kmax) from vecchia_group_classes (one launch per class).  Returns (out, status) on
    the device, as vecchia_loglik_grad_info."""
    import torch
    for t, dt, nm_ in ((locs, torch.float64, "locs"), (y, torch.float64, "y"),
                       (X, torch.float64, "X"), (block_off, torch.int64, "block_off"),
                       (block_idx, torch.int32, "block_idx"), (nmemb, torch.int32, "nmemb"),
                       (covparms, torch.float64, "covparms")):
        _dev_tensor_check(t, dt, nm_)
    n, d = locs.shape
    p = X.shape[1]
    q = nparms(covfun, d)
    ng = nmemb.shape[0]
    if classes is None:
        gptr, nclass = None, 1
        class_off = np.array([0, ng], dtype=np.int64)
        class_kmax = np.array([int(kmax)], dtype=np.int32)
    else:
        gorder, class_off, class_kmax = classes
        _dev_tensor_check(gorder, torch.int32, "gorder")
        gptr, nclass = _dptr(gorder), len(class_kmax)
        class_off = np.ascontiguousarray(class_off, dtype=np.int64)
        class_kmax = np.ascontiguousarray(class_kmax, dtype=np.int32)
    dev = locs.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    if out is None:
        out = torch.empty(1 + q + q * q + p, dtype=torch.float64, device=dev)
    if status is None:
        status = torch.empty(2, dtype=torch.int64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    P = ctypes.c_void_p
    _check(lib().vecchia_grouped_loglik_grad_info(
        handle.ptr, _dptr(locs), _dptr(y), _dptr(X), n, d, p, ng, _dptr(block_off),
        _dptr(block_idx), _dptr(nmemb), gptr, nclass, class_off.ctypes.data_as(P),
        class_kmax.ctypes.data_as(P), _dptr(covparms), covfun, _PREC[prec],
        ctypes.c_void_p(stream.cuda_stream), _dptr(out), _dptr(status)))
    return out, status


def vecchia_measure_peaks(handle: Handle | None = None, device: int = 0) -> dict:
    """Measured FP64 / FP32 FMA-chain GFLOP/s, covariance evaluations per second and the
    FP64 tensor-core GFLOP/s on the device (see vecchia_measure_peaks in include/vecchia.h)."""
    if handle is None:
        handle = default_handle(device)
    out = (ctypes.c_double * 5)()
    _check(lib().vecchia_measure_peaks(handle.ptr, ctypes.cast(out, ctypes.c_void_p)))
    return {"fp64_gflops": out[0], "fp32_gflops": out[1], "exp_pairs_per_s": out[2],
            "matern_pairs_per_s": out[3], "fp64_tensor_gflops": out[4]}


def vecchia_covariance_pairs(covfun: int, covparms, la, lb, same, stream=None,
                             handle: Handle | None = None):
    """Device covariance C (npairs,) and dC (npairs, q) for CUDA tensors la, lb (npairs, d)."""
    import torch
    _dev_tensor_check(covparms, torch.float64, "covparms")
    _dev_tensor_check(la, torch.float64, "la")
    _dev_tensor_check(lb, torch.float64, "lb")
    _dev_tensor_check(same, torch.int32, "same")
    npairs, d = la.shape
    q = nparms(covfun, d)
    dev = la.device
    if handle is None:
        handle = default_handle(dev.index if dev.index is not None else 0)
    C = torch.empty(npairs, dtype=torch.float64, device=dev)
    dC = torch.empty(npairs, q, dtype=torch.float64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    _check(lib().vecchia_covariance_pairs(handle.ptr, covfun, _dptr(covparms), d, npairs,
                                          _dptr(la), _dptr(lb), _dptr(same), _dptr(C), _dptr(dC),
                                          ctypes.c_void_p(stream.cuda_stream)))
    return C, dC

"""CPU FP64 oracle for the Vecchia likelihood pass -- TEST INFRASTRUCTURE.

Only the tests, the smoke check (``__graft_entry__.smoke``) and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports, links or calls it
and shares no code with it; the oracle is the independent reference the CUDA path is
checked against.

Every function follows the paper (James & Guinness, arXiv 2407.02740):
  * ``stats`` / ``records``  -- Algorithm 1, per-observation sums (Sec. 3), with the
    elided derivative half written out from the Cholesky differential (see the C file).
  * ``profile``              -- the "separate function" of Sec. 3: profiled beta,
    loglikelihood, gradient and Fisher information.
  * ``loglik_grad_info``     -- both of the above.
  * ``fisher_fit``           -- Fisher scoring, Eq. 4, on log-parameters.
  * ``cov_pairs``            -- the covariance functions of Sec. 4.3 (Eq. 6: isotropic, and
    with one range per coordinate) and Matern.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vecchia_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

EXP_ISO, MATERN_ISO, EXP_SPACETIME, EXP_ANISO = 0, 1, 2, 3
NPARMS = {EXP_ISO: 3, MATERN_ISO: 4, EXP_SPACETIME: 4}   # families with a fixed count
DMAX_ANISO = 20


def nparms(covfun: int, d: int) -> int:
    """Number of covariance parameters of a family in d dimensions: the anisotropic
    exponential has one range per coordinate, theta = (sigma2, rho_1..rho_d, tau2)."""
    if covfun == EXP_ANISO:
        if not 1 <= d <= DMAX_ANISO:
            raise ValueError("anisotropic exponential: d must be in [1, %d]" % DMAX_ANISO)
        return d + 2
    return NPARMS[covfun]
STATUS = {0: "ok", 1: "bad argument", 2: "not positive definite", 3: "non-finite",
          4: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (code %d)" % (what, STATUS.get(code, "?"), code))
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -fopenmp, no FMA contraction) in-tree."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-std=gnu11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_nparms.argtypes = [ci]
        lib.orc_nparms_d.argtypes = [ci, ci]
        lib.orc_stats_len.argtypes = [ci, ci]
        lib.orc_cov_pairs.argtypes = [ci, ci, P, i64, P, P, P, P, P]
        lib.orc_psi.argtypes = [cd]
        lib.orc_psi.restype = cd
        lib.orc_vecchia_stats.argtypes = [P, P, P, P, i64, ci, ci, ci, P, ci, P, P, ci]
        lib.orc_vecchia_records.argtypes = [P, P, P, P, i64, ci, ci, ci, P, ci, P]
        lib.orc_profile.argtypes = [P, i64, ci, ci, P, P, P, P]
        lib.orc_loglik_grad_info.argtypes = [P, P, P, P, i64, ci, ci, ci, P, ci, P, P, P, P,
                                             P, ci]
        lib.orc_fisher_fit.argtypes = [P, P, P, P, i64, ci, ci, ci, ci, P, cd, ci, P, P, P, P,
                                       P, P, P, ci]
        for f in (lib.orc_nparms, lib.orc_nparms_d, lib.orc_stats_len, lib.orc_cov_pairs, lib.orc_vecchia_stats,
                  lib.orc_vecchia_records, lib.orc_profile, lib.orc_loglik_grad_info,
                  lib.orc_fisher_fit):
            f.restype = ci
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _inputs(locs, y, X, NN):
    locs = np.ascontiguousarray(locs, dtype=np.float64)
    if locs.ndim == 1:
        locs = locs[:, None]
    y = np.ascontiguousarray(y, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    NN = np.ascontiguousarray(NN, dtype=np.int32)
    n, d = locs.shape
    if y.shape != (n,) or X.shape[0] != n or NN.shape[0] != n:
        raise ValueError("inconsistent input shapes")
    return locs, y, X, NN, n, d, X.shape[1], NN.shape[1] - 1


def stats_len(p: int, q: int) -> int:
    return 2 + p * p + p + q * (2 + p * p + p) + q * q


def split_stats(s: np.ndarray, p: int, q: int) -> dict:
    """Names the fields of an Algorithm 1 record (see the C file for the layout)."""
    o = 0
    out = {}
    for name, shape in (("logdet", ()), ("ySy", ()), ("XSX", (p, p)), ("ySX", (p,)),
                        ("dlogdet", (q,)), ("dySy", (q,)), ("dXSX", (q, p, p)),
                        ("dySX", (q, p)), ("ainfo", (q, q))):
        size = int(np.prod(shape)) if shape else 1
        out[name] = s[..., o:o + size].reshape(s.shape[:-1] + shape)
        o += size
    return out


def cov_pairs(covfun, theta, la, lb, same):
    """Covariance C and its theta-derivatives dC (npairs x q) for location pairs."""
    la = np.ascontiguousarray(la, dtype=np.float64)
    lb = np.ascontiguousarray(lb, dtype=np.float64)
    if la.ndim == 1:
        la, lb = la[:, None], lb[:, None]
    same = np.ascontiguousarray(same, dtype=np.int32)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    npairs, d = la.shape
    q = nparms(covfun, d)
    C = np.empty(npairs)
    dC = np.empty((npairs, q))
    rc = _load().orc_cov_pairs(covfun, d, _p(theta), npairs, _p(la), _p(lb), _p(same), _p(C),
                               _p(dC))
    if rc:
        raise OracleError(rc, "cov_pairs")
    return C, dC


def digamma(x: float) -> float:
    return _load().orc_psi(float(x))


def stats(locs, y, X, NN, theta, covfun, nthreads: int = 0):
    """Summed Algorithm 1 record.  Returns (record, bad_index)."""
    locs, y, X, NN, n, d, p, m = _inputs(locs, y, X, NN)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    q = nparms(covfun, d)
    out = np.empty(stats_len(p, q))
    bad = ctypes.c_int64(-1)
    rc = _load().orc_vecchia_stats(_p(locs), _p(y), _p(X), _p(NN), n, d, p, m, _p(theta),
                                   covfun, _p(out), ctypes.byref(bad), nthreads)
    if rc:
        err = OracleError(rc, "vecchia stats")
        err.bad_index = bad.value
        raise err
    return out, bad.value


def records(locs, y, X, NN, theta, covfun):
    """Per-observation Algorithm 1 records (n x S), for tiny inputs."""
    locs, y, X, NN, n, d, p, m = _inputs(locs, y, X, NN)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    q = nparms(covfun, d)
    out = np.empty((n, stats_len(p, q)))
    rc = _load().orc_vecchia_records(_p(locs), _p(y), _p(X), _p(NN), n, d, p, m, _p(theta),
                                     covfun, _p(out))
    if rc:
        raise OracleError(rc, "vecchia records")
    return out


def profile(rec, n, p, q):
    rec = np.ascontiguousarray(rec, dtype=np.float64)
    ll = ctypes.c_double()
    grad = np.empty(q)
    info = np.empty((q, q))
    beta = np.empty(p)
    rc = _load().orc_profile(_p(rec), n, p, q, ctypes.byref(ll), _p(grad), _p(info), _p(beta))
    if rc:
        raise OracleError(rc, "profile")
    return ll.value, grad, info, beta


def loglik_grad_info(locs, y, X, NN, theta, covfun, nthreads: int = 0):
    """Profiled-beta Vecchia loglikelihood, gradient, Fisher information and betahat."""
    locs, y, X, NN, n, d, p, m = _inputs(locs, y, X, NN)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    q = nparms(covfun, d)
    ll = ctypes.c_double()
    grad = np.empty(q)
    info = np.empty((q, q))
    beta = np.empty(p)
    bad = ctypes.c_int64(-1)
    rc = _load().orc_loglik_grad_info(_p(locs), _p(y), _p(X), _p(NN), n, d, p, m, _p(theta),
                                      covfun, ctypes.byref(ll), _p(grad), _p(info), _p(beta),
                                      ctypes.byref(bad), nthreads)
    if rc:
        err = OracleError(rc, "loglik_grad_info")
        err.bad_index = bad.value
        raise err
    return {"loglik": ll.value, "grad": grad, "info": info, "betahat": beta,
            "bad_index": bad.value}


def fisher_fit(locs, y, X, NN, covfun, start, tol: float = 1e-4, maxit: int = 40,
               nthreads: int = 0):
    """Fisher scoring on log theta (Eq. 4) with step halving; see the C file for rules."""
    locs, y, X, NN, n, d, p, m = _inputs(locs, y, X, NN)
    start = np.ascontiguousarray(start, dtype=np.float64)
    q = nparms(covfun, d)
    theta = np.empty(q)
    beta = np.empty(p)
    ll = ctypes.c_double()
    grad = np.empty(q)
    info = np.empty((q, q))
    iters = ctypes.c_int()
    status = ctypes.c_int()
    rc = _load().orc_fisher_fit(_p(locs), _p(y), _p(X), _p(NN), n, d, p, m, covfun, _p(start),
                                tol, maxit, _p(theta), _p(beta), ctypes.byref(ll), _p(grad),
                                _p(info), ctypes.byref(iters), ctypes.byref(status), nthreads)
    if rc:
        raise OracleError(rc, "fisher_fit")
    return {"theta": theta, "betahat": beta, "loglik": ll.value, "grad": grad, "info": info,
            "iters": iters.value, "status": status.value}

"""Seeded synthetic workloads for the Vecchia likelihood pass.

This module is input generation only.  It is shared by the two sides that consume the
inputs -- the CPU oracle (``oracle/``) and the CUDA library (``paper_2407_02740_gb300``)
-- and it imports neither.  It computes the maxmin ordering and the ordered
nearest-neighbour array (``NNarray``) once, so both sides receive identical arrays
(Sec. 2.1 and Sec. 3 of the paper: ordering, then ``NNarray``, then the fit).

To give the synthetic fields the statistical structure of the paper's data, the
generators draw ``y`` from a Gaussian process.  That needs a covariance function, so
this module carries its own small one (numpy closed forms for exponential and
half-integer Matern, ``scipy.special.kv`` otherwise).  Neither the oracle nor the CUDA
library uses it for anything they compute.

Workloads (the recipes stand in for the paper's datasets, which are not available):

* ``cfg_small_exp``  -- n = 2000 uniform in [0,1]^2, exponential (1, 0.1, 0.01), X = 1,
  dense-Cholesky draw, maxmin order, m = 10.  One evaluation at the true parameters.
* ``cfg_matern_100k`` -- n = 100000 uniform in [0,1]^2, Matern (2.0, 0.05, 1.5, 0.05),
  X = [1, x1, x2], beta = (1, 0.5, -0.5), sequential draw with m = 60, fit with m = 30
  from (var y, 0.1, 1, 0.1).  Stands in for the Jason-3 subset runs (Table 1, Fig. 5).
* ``cfg_swath_1m2``  -- 16 time slices x 8 swath bands x 9375 points = 1.2M points
  (lon, lat, time); space-time exponential (1, 5 deg, 2 slices, 0.1); X = [1, lat];
  sequential draw with m = 40; fit with m = 30.  Stands in for "Jason-3 + Time" (Table 2).
* ``cfg_elevators_like`` -- n = 15000 points with 18 N(0,1) attributes as locations,
  exponential with one range per attribute (log-spaced 1..8), X = 1; sequential draw
  with m = 30; fit with m = 10 or 30.  Stands in for Elevators (Table 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prep.c")
_LIB = os.path.join(_HERE, "libprep.so")

EXP_ISO = 0
MATERN_ISO = 1
EXP_SPACETIME = 2
EXP_ANISO = 3          # one range per coordinate: theta = (sigma2, rho_1..rho_d, tau2)
NPARMS = {EXP_ISO: 3, MATERN_ISO: 4, EXP_SPACETIME: 4}


def build(force: bool = False) -> str:
    """Compile the preprocessing library in-tree (gcc, plain C, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-std=gnu11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        lib.prep_maxmin.argtypes = [P, i64, ci, P]
        lib.prep_maxmin_brute.argtypes = [P, i64, ci, P]
        lib.prep_ordered_nn.argtypes = [P, i64, ci, ci, P]
        lib.prep_ordered_nn_brute.argtypes = [P, i64, ci, ci, P]
        lib.prep_seq_recurrence.argtypes = [i64, ci, P, P, P, P, P]
        lib.prep_seq_weights.argtypes = [i64, ci, ci, P, P, ci, P, P, P]
        lib.prep_seq_weights.restype = ci
        for f in (lib.prep_maxmin, lib.prep_maxmin_brute, lib.prep_ordered_nn,
                  lib.prep_ordered_nn_brute, lib.prep_seq_recurrence):
            f.restype = ci
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def maxmin_order(x: np.ndarray, brute: bool = False) -> np.ndarray:
    """Exact maxmin ordering of the rows of x (n x d); returns original indices.  More
    than 3 coordinates always take the O(n^2 d) search."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    out = np.empty(n, dtype=np.int64)
    f = _load().prep_maxmin_brute if (brute or d > 3) else _load().prep_maxmin
    rc = f(_ptr(x), n, d, _ptr(out))
    if rc != 0:
        raise RuntimeError("maxmin ordering failed (code %d)" % rc)
    return out


def ordered_nn(x: np.ndarray, m: int, brute: bool = False) -> np.ndarray:
    """NNarray (n x (m+1), int32): row i = [i, nearest earlier points..., -1 padding]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    out = np.empty((n, m + 1), dtype=np.int32)
    f = _load().prep_ordered_nn_brute if (brute or d > 3) else _load().prep_ordered_nn
    rc = f(_ptr(x), n, d, m, _ptr(out))
    if rc != 0:
        raise RuntimeError("ordered NN failed (code %d)" % rc)
    return out


# ------------------------------------------------------------------------------------
# Generator-side covariance (for drawing y only)
# ------------------------------------------------------------------------------------
def _gen_corr(covfun: int, theta, la: np.ndarray, lb: np.ndarray) -> np.ndarray:
    """Correlation (without sigma2 and nugget) between location arrays la, lb (..., d)."""
    diff = la - lb
    if covfun == EXP_ANISO:
        rho = np.asarray(theta[1:-1], dtype=np.float64)
        return np.exp(-np.sqrt(np.sum((diff / rho) ** 2, axis=-1)))
    if covfun == EXP_SPACETIME:
        D = np.sqrt((diff[..., 0] ** 2 + diff[..., 1] ** 2) / theta[1] ** 2
                    + diff[..., 2] ** 2 / theta[2] ** 2)
        return np.exp(-D)
    x = np.sqrt(np.sum(diff * diff, axis=-1)) / theta[1]
    if covfun == EXP_ISO:
        return np.exp(-x)
    nu = float(theta[2])
    if nu == 0.5:
        return np.exp(-x)
    if nu == 1.5:
        return (1.0 + x) * np.exp(-x)
    if nu == 2.5:
        return (1.0 + x + x * x / 3.0) * np.exp(-x)
    from scipy.special import gamma, kv
    out = np.ones_like(x)
    pos = x > 0
    xp = x[pos]
    out[pos] = 2.0 ** (1.0 - nu) / gamma(nu) * xp ** nu * kv(nu, xp)
    return out


def _gen_cov_block(covfun, theta, locs_blk):
    """Full covariance of a block of locations (..., K, d), nugget on the diagonal."""
    R = _gen_corr(covfun, theta, locs_blk[..., :, None, :], locs_blk[..., None, :, :])
    tau2 = theta[-1]
    K = locs_blk.shape[-2]
    return theta[0] * (R + tau2 * np.eye(K))


def simulate_dense(covfun, theta, locs, rng) -> np.ndarray:
    """Zero-mean draw with covariance sigma2 (R + tau2 I), by dense Cholesky."""
    import scipy.linalg
    S = _gen_cov_block(covfun, theta, locs)
    Lc = scipy.linalg.cholesky(S, lower=True)
    return Lc @ rng.standard_normal(locs.shape[0])


def simulate_sequential(covfun, theta, locs, NN, rng, chunk: int = 2048) -> np.ndarray:
    """Zero-mean draw from the sequential (Vecchia) model defined by NN:
    e_i = w_i^T e_{N(i)} + sqrt(v_i) z_i with w_i, v_i the conditional regression of the
    Gaussian process on the listed earlier neighbours."""
    n, W = NN.shape
    m = W - 1
    Wt = np.zeros((n, max(m, 1)), dtype=np.float64)
    sd = np.zeros(n, dtype=np.float64)
    # closed-form kernels: the C helper (OpenMP); other smoothness values: numpy + scipy
    kind = None
    th = np.asarray(theta, dtype=np.float64)
    if covfun == EXP_ISO:
        kind, thc = 0, th[[0, 1, 2]]
    elif covfun == EXP_ANISO:
        # the exponential on coordinates divided by their ranges
        locs = np.asarray(locs, dtype=np.float64) / th[1:-1]
        kind, thc = 0, np.array([th[0], 1.0, th[-1]])
    elif covfun == EXP_SPACETIME:
        kind, thc = 3, th
    elif covfun == MATERN_ISO and float(th[2]) in (0.5, 1.5, 2.5):
        kind = {0.5: 0, 1.5: 1, 2.5: 2}[float(th[2])]
        thc = th[[0, 1, 3]]
    if kind is not None:
        NNc = np.ascontiguousarray(NN, dtype=np.int32)
        Wc = np.zeros((n, max(m, 1)))
        locs_c = np.ascontiguousarray(locs, dtype=np.float64)
        thc = np.ascontiguousarray(thc, dtype=np.float64)
        rc = _load().prep_seq_weights(n, locs_c.shape[1], m, _ptr(NNc), _ptr(locs_c), kind,
                                      _ptr(thc), _ptr(Wc), _ptr(sd))
        if rc != 0:
            raise RuntimeError("sequential weights failed (block not positive definite)")
        Wt = Wc
    kcount = (NN[:, 1:] >= 0).sum(axis=1) if m > 0 else np.zeros(n, dtype=np.int64)
    for k in (np.unique(kcount) if kind is None else []):
        idx = np.nonzero(kcount == k)[0]
        for s in range(0, len(idx), chunk):
            ii = idx[s:s + chunk]
            if k == 0:
                sd[ii] = np.sqrt(theta[0] * (1.0 + theta[-1]))
                continue
            nb = NN[ii, 1:1 + k]                      # (B, k)
            blk = np.concatenate([locs[nb], locs[ii][:, None, :]], axis=1)  # (B, k+1, d)
            S = _gen_cov_block(covfun, theta, blk)
            Snn = S[:, :k, :k]
            sni = S[:, :k, k]
            w = np.linalg.solve(Snn, sni[..., None])[..., 0]
            v = S[:, k, k] - np.einsum("bi,bi->b", sni, w)
            Wt[ii, :k] = w
            sd[ii] = np.sqrt(np.maximum(v, 0.0))
    z = rng.standard_normal(n)
    e = np.empty(n, dtype=np.float64)
    NNc = np.ascontiguousarray(NN, dtype=np.int32)
    Wc = np.ascontiguousarray(Wt[:, :m] if m > 0 else np.zeros((n, 0)))
    rc = _load().prep_seq_recurrence(n, m, _ptr(NNc), _ptr(Wc), _ptr(sd), _ptr(z), _ptr(e))
    if rc != 0:
        raise RuntimeError("sequential recurrence failed")
    return e


# ------------------------------------------------------------------------------------
# Workloads
# ------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    covfun: int
    locs: np.ndarray        # n x d, float64, maxmin order
    y: np.ndarray           # n, float64
    X: np.ndarray           # n x p, float64
    NN: np.ndarray          # n x (m+1), int32
    theta_true: np.ndarray  # q
    theta_start: np.ndarray  # q
    m: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.locs.shape[0]

    @property
    def d(self):
        return self.locs.shape[1]

    @property
    def p(self):
        return self.X.shape[1]


def _finish(name, covfun, locs, y, X, m, theta_true, theta_start, NN=None, **meta):
    if NN is None:
        NN = ordered_nn(meta.pop("nn_coords", locs), m)
    else:
        meta.pop("nn_coords", None)
    return Workload(name=name, covfun=covfun,
                    locs=np.ascontiguousarray(locs, dtype=np.float64),
                    y=np.ascontiguousarray(y, dtype=np.float64),
                    X=np.ascontiguousarray(X, dtype=np.float64),
                    NN=np.ascontiguousarray(NN, dtype=np.int32),
                    theta_true=np.asarray(theta_true, dtype=np.float64),
                    theta_start=np.asarray(theta_start, dtype=np.float64), m=m, meta=meta)


def make_field(n: int, covfun: int, theta, m: int, p: int = 1, seed: int = 0,
               sim: str = "dense", m_sim: int | None = None, d: int = 2,
               beta=None, ordering: str = "maxmin", name: str = "field") -> Workload:
    """Generic seeded field in [0,1]^d (d=3 for the space-time covariance, d = len(theta)-2
    for the anisotropic exponential, whose ordering and neighbours are taken on the
    coordinates divided by the ranges), used by tests.
    X columns: 1, then the first p-1 coordinates.  sim = 'dense' or 'sequential'."""
    rng = np.random.default_rng(seed)
    if covfun == EXP_SPACETIME:
        d = 3
    if covfun == EXP_ANISO:
        d = len(theta) - 2
    scale = (1.0 / np.asarray(theta[1:-1], dtype=np.float64)) if covfun == EXP_ANISO else 1.0
    locs = rng.uniform(0.0, 1.0, size=(n, d))
    if ordering == "maxmin":
        locs = locs[maxmin_order(locs * scale)]
    X = np.ones((n, p))
    for c in range(1, p):
        X[:, c] = locs[:, (c - 1) % d]
    beta = np.zeros(p) if beta is None else np.asarray(beta, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    if sim == "dense":
        e = simulate_dense(covfun, theta, locs, rng)
    else:
        ms = m if m_sim is None else m_sim
        e = simulate_sequential(covfun, theta, locs, ordered_nn(locs * scale, ms), rng)
    y = X @ beta + e
    start = theta.copy()
    return _finish(name, covfun, locs, y, X, m, theta, start, seed=seed, nn_coords=locs * scale)


def cfg_small_exp(seed: int = 1001) -> Workload:
    """n=2000 in [0,1]^2, exponential (sigma2, rho, tau2) = (1, 0.1, 0.01), X = 1, beta = 0,
    dense-Cholesky draw, maxmin order, m = 10."""
    rng = np.random.default_rng(seed)
    n, m = 2000, 10
    theta = np.array([1.0, 0.1, 0.01])
    locs = rng.uniform(0.0, 1.0, size=(n, 2))
    locs = locs[maxmin_order(locs)]
    y = simulate_dense(EXP_ISO, theta, locs, rng)
    X = np.ones((n, 1))
    start = np.array([np.var(y), 0.2, 0.1])
    return _finish("exp_n2000_m10", EXP_ISO, locs, y, X, m, theta, start, seed=seed)


def cfg_matern_100k(seed: int = 1002, n: int = 100_000, m: int = 30, m_sim: int = 60
                    ) -> Workload:
    """n=1e5 in [0,1]^2, Matern (2.0, 0.05, 1.5, 0.05), X = [1, x1, x2],
    beta = (1, 0.5, -0.5), sequential draw with m_sim = 60, fit m = 30,
    start (var y, 0.1, 1, 0.1)."""
    rng = np.random.default_rng(seed)
    theta = np.array([2.0, 0.05, 1.5, 0.05])
    locs = rng.uniform(0.0, 1.0, size=(n, 2))
    locs = locs[maxmin_order(locs)]
    NN60 = ordered_nn(locs, m_sim)
    e = simulate_sequential(MATERN_ISO, theta, locs, NN60, rng)
    X = np.column_stack([np.ones(n), locs[:, 0], locs[:, 1]])
    beta = np.array([1.0, 0.5, -0.5])
    y = X @ beta + e
    NN = np.ascontiguousarray(NN60[:, : m + 1])
    start = np.array([np.var(y), 0.1, 1.0, 0.1])
    return _finish("matern_n%d_m%d" % (n, m), MATERN_ISO, locs, y, X, m, theta, start,
                   NN=NN, seed=seed, m_sim=m_sim)


def swath_locations(rng, slices: int = 16, bands: int = 8, per: int = 9375) -> np.ndarray:
    """Satellite-like (lon, lat, time): band b of slice t follows
    lon = (45 b + 7.5 t + 360 s) mod 360, lat = clip(60 sin(2 pi s + b), -60, 60),
    s ~ U[0,1), plus N(0, 0.5 deg) jitter on both, time = t + 0.1 U."""
    out = []
    for t in range(slices):
        for b in range(bands):
            s = rng.uniform(0.0, 1.0, size=per)
            lon = np.mod(45.0 * b + 7.5 * t + 360.0 * s, 360.0) + rng.normal(0.0, 0.5, per)
            lat = np.clip(60.0 * np.sin(2 * np.pi * s + b), -60.0, 60.0) + rng.normal(0.0, 0.5, per)
            tim = t + 0.1 * rng.uniform(0.0, 1.0, size=per)
            out.append(np.column_stack([lon, lat, tim]))
    return np.concatenate(out, axis=0)


def cfg_swath_1m2(seed: int = 1003, slices: int = 16, bands: int = 8, per: int = 9375,
                  m: int = 30, m_sim: int = 40) -> Workload:
    """Space-time exponential (1, 5, 2, 0.1) on swath locations, X = [1, lat],
    beta = (1, 0.01), sequential draw with m_sim = 40, fit m = 30."""
    rng = np.random.default_rng(seed)
    theta = np.array([1.0, 5.0, 2.0, 0.1])
    locs = swath_locations(rng, slices, bands, per)
    scaled = locs / np.array([theta[1], theta[1], theta[2]])
    order = maxmin_order(scaled)
    locs = locs[order]
    scaled = scaled[order]
    NNs = ordered_nn(scaled, m_sim)
    e = simulate_sequential(EXP_SPACETIME, theta, locs, NNs, rng)
    X = np.column_stack([np.ones(locs.shape[0]), locs[:, 1]])
    y = X @ np.array([1.0, 0.01]) + e
    NN = np.ascontiguousarray(NNs[:, : m + 1]) if m <= m_sim else ordered_nn(scaled, m)
    start = np.array([np.var(y), 10.0, 4.0, 0.1])
    return _finish("swath_n%d_m%d" % (locs.shape[0], m), EXP_SPACETIME, locs, y, X, m, theta,
                   start, NN=NN, seed=seed, m_sim=m_sim)


def grouped_order(locs: np.ndarray, g: int, gmax: int | None = None):
    """An ordering for grouped conditioning: spatially compact groups of about g points
    (the cells of a cubic grid over the coordinates, cells of more than gmax points split
    into runs of gmax), the groups in the maxmin order of their centroids, each group's
    points by index.  Returns (order, group_off): group b is order[group_off[b] :
    group_off[b + 1]], a contiguous range of the ordering."""
    locs = np.asarray(locs, dtype=np.float64)
    n, d = locs.shape
    gmax = 2 * g if gmax is None else gmax
    xy = locs
    lo, hi = xy.min(axis=0), xy.max(axis=0)
    ncell = max(1, int(round((n / g) ** (1.0 / d))))
    cid = np.minimum(((xy - lo) / np.maximum(hi - lo, 1e-300) * ncell).astype(np.int64), ncell - 1)
    key = np.zeros(n, dtype=np.int64)
    for k in range(d):
        key = key * ncell + cid[:, k]
    by_cell = np.argsort(key, kind="stable")
    bounds = np.flatnonzero(np.diff(key[by_cell])) + 1
    groups = []
    for cell in np.split(by_cell, bounds):
        for s in range(0, len(cell), gmax):
            groups.append(np.sort(cell[s:s + gmax]))
    cent = np.array([xy[gr].mean(axis=0) for gr in groups])
    gorder = maxmin_order(cent)
    order = np.concatenate([groups[k] for k in gorder])
    off = np.zeros(len(groups) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(groups[k]) for k in gorder])
    return order, off


def grouped_field(n: int, covfun: int, theta, m: int, g: int, p: int = 1, seed: int = 0,
                  m_sim: int = 30, beta=None, gmax: int | None = None):
    """A field in [0,1]^2 (d = 3 for the space-time covariance) in a grouped ordering
    (grouped_order, groups of about g, at most gmax), y from a sequential draw with m_sim
    neighbours in that ordering, NNarray with m.  Returns (Workload, group_off)."""
    rng = np.random.default_rng(seed)
    d = 3 if covfun == EXP_SPACETIME else 2
    locs = rng.uniform(0.0, 1.0, size=(n, d))
    order, goff = grouped_order(locs, g, gmax)
    locs = locs[order]
    X = np.ones((n, p))
    for c in range(1, p):
        X[:, c] = locs[:, (c - 1) % d]
    beta = np.zeros(p) if beta is None else np.asarray(beta, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    NNs = ordered_nn(locs, max(m, m_sim))
    e = simulate_sequential(covfun, theta, locs, NNs[:, :m_sim + 1], rng)
    y = X @ beta + e
    w = _finish("grouped_n%d_g%d_m%d" % (n, g, m), covfun, locs, y, X, m, theta, theta.copy(),
                NN=np.ascontiguousarray(NNs[:, :m + 1]), seed=seed, g=g)
    return w, goff


def elevators_ranges(d: int = 18) -> np.ndarray:
    """Ranges of the Elevators-like field: log-spaced from 1 to 8 (standardised attributes),
    so the attributes differ in relevance by a factor of 8 and every range stays
    identifiable (with ranges up to 30 the least relevant ones drift to infinity in a fit)."""
    return np.exp(np.linspace(np.log(1.0), np.log(8.0), d))


def cfg_elevators_like(seed: int = 1010, n: int = 15000, d: int = 18, m: int = 30,
                       m_sim: int = 30) -> Workload:
    """Stands in for the Elevators runs (n = 15k training points, 18 attributes used as
    locations, exponential covariance with one range per attribute, X = 1): attributes
    i.i.d. N(0, 1) (standardised), theta = (1, ranges, 0.1), sequential draw with
    m_sim = 30, beta = 0.5.  Ordering and neighbours are taken on the attributes divided
    by the true ranges.  The fit starts from (var y, 2, ..., 2, 0.2)."""
    rng = np.random.default_rng(seed)
    rho = elevators_ranges(d)
    theta = np.concatenate([[1.0], rho, [0.1]])
    locs = rng.standard_normal((n, d))
    scaled = locs / rho
    order = maxmin_order(scaled)
    locs = locs[order]
    scaled = scaled[order]
    NNs = ordered_nn(scaled, max(m, m_sim))
    e = simulate_sequential(EXP_ANISO, theta, locs, NNs[:, : m_sim + 1], rng)
    X = np.ones((n, 1))
    y = 0.5 + e
    NN = np.ascontiguousarray(NNs[:, : m + 1])
    start = np.concatenate([[np.var(y)], np.full(d, 2.0), [0.2]])
    return _finish("elevators_like_n%d_d%d_m%d" % (n, d, m), EXP_ANISO, locs, y, X, m, theta,
                   start, NN=NN, seed=seed, m_sim=m_sim)


@dataclass
class BatchWorkload:
    """Many independent fields, concatenated: dataset b owns rows off[b]:off[b+1] of locs,
    y, X and a block of NN (its own n_b x (m_b+1) array, indices local to the dataset)."""
    covfun: int
    locs: np.ndarray
    y: np.ndarray
    X: np.ndarray
    NN: np.ndarray          # flat int32, concatenated per-dataset arrays
    offsets: np.ndarray     # nbatch + 1, int64
    m: np.ndarray           # nbatch, int32
    theta_true: np.ndarray  # nbatch x q
    theta_start: np.ndarray  # nbatch x q

    @property
    def nbatch(self):
        return len(self.m)

    def dataset(self, b) -> Workload:
        s, e = self.offsets[b], self.offsets[b + 1]
        nn_s = int(sum((self.offsets[k + 1] - self.offsets[k]) * (self.m[k] + 1) for k in range(b)))
        nb, mb = e - s, int(self.m[b])
        NN = self.NN[nn_s: nn_s + nb * (mb + 1)].reshape(nb, mb + 1)
        return Workload("batch%d" % b, self.covfun, self.locs[s:e], self.y[s:e], self.X[s:e], NN,
                        self.theta_true[b], self.theta_start[b], mb)


def cfg_batch(seed: int = 1004, nbatch: int = 256, n_range=(1000, 50000), m_choices=(10, 20, 40),
              nu_choices=(0.5, 1.5, 2.5), m_sim: int = 40) -> BatchWorkload:
    """nbatch Matern fields in [0,1]^2: n log-uniform in n_range, m from m_choices,
    sigma2 log-uniform [0.5, 2], rho log-uniform [0.02, 0.3], nu from nu_choices, tau2
    log-uniform [0.001, 0.2], X = 1, beta = 0, sequential draw with m_sim neighbours.
    Dataset b draws from its own generator (child b of SeedSequence(seed)), so the
    datasets are built in parallel threads (the C helpers release the GIL) and do not
    depend on the thread schedule."""
    from concurrent.futures import ThreadPoolExecutor
    lo, hi = np.log(n_range[0]), np.log(n_range[1])
    children = np.random.SeedSequence(seed).spawn(nbatch)

    def one(b):
        rng = np.random.default_rng(children[b])
        n = int(round(np.exp(rng.uniform(lo, hi))))
        m = int(rng.choice(m_choices))
        theta = np.array([np.exp(rng.uniform(np.log(0.5), np.log(2.0))),
                          np.exp(rng.uniform(np.log(0.02), np.log(0.3))),
                          float(rng.choice(nu_choices)),
                          np.exp(rng.uniform(np.log(0.001), np.log(0.2)))])
        L = rng.uniform(0.0, 1.0, size=(n, 2))
        L = L[maxmin_order(L)]
        NNsim = ordered_nn(L, max(m, m_sim))
        e = simulate_sequential(MATERN_ISO, theta, L, NNsim[:, : m_sim + 1], rng)
        return (L, e, np.ones((n, 1)), np.ascontiguousarray(NNsim[:, : m + 1]).ravel(), m, theta,
                np.array([np.var(e), 0.1, 1.0, 0.1]))

    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        parts = list(ex.map(one, range(nbatch)))
    locs, ys, Xs, NNs, ms, th, st = (list(t) for t in zip(*parts))
    off = np.concatenate([[0], np.cumsum([len(e) for e in ys])])
    return BatchWorkload(MATERN_ISO, np.concatenate(locs), np.concatenate(ys), np.concatenate(Xs),
                         np.concatenate(NNs).astype(np.int32), np.array(off, dtype=np.int64),
                         np.array(ms, dtype=np.int32), np.array(th), np.array(st))

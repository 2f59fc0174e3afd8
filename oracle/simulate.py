"""Oracle for the sequential Vecchia draw -- TEST INFRASTRUCTURE (see ``oracle/__init__``).

The Vecchia joint density (Sec. 2.1, Eq. 3) is the product over the ordering of the
conditional densities p(y_i | y_N(i)), N(i) the listed earlier neighbours of i.  Under the
Gaussian covariance model each conditional is Gaussian with mean w_i' y_N(i) and variance
v_i, the regression of y_i on y_N(i):

    w_i = Sigma_NN^-1 Sigma_Ni,    v_i = Sigma_ii - Sigma_iN w_i,

(nugget included on the diagonal, as in the likelihood).  A draw takes the ordering in
turn: y_i = w_i' y_N(i) + sqrt(v_i) z_i.  Written as a row of a sparse inverse factor,
b_i = (1, -w_i) / sqrt(v_i) on (i, N(i)) gives b_i . (y_i, y_N(i)) = z_i.

Covariances come from the oracle's own covariance functions (``cov_pairs``); the solves
are numpy FP64 (numpy.linalg.solve).  Loops are plain Python: small inputs only.
"""
from __future__ import annotations

import numpy as np

from . import cov_pairs, nparms


def _cov_matrix(covfun, theta, pts):
    """Dense covariance of the points pts (k x d), nugget on the diagonal."""
    k = len(pts)
    ia, ib = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    la = pts[ia.ravel()]
    lb = pts[ib.ravel()]
    same = (ia.ravel() == ib.ravel()).astype(np.int32)
    C, _ = cov_pairs(covfun, theta, la, lb, same)
    return C.reshape(k, k)


def factor_rows(locs, NN, theta, covfun):
    """Rows b_i (n x (m+1), NNarray order: entry 0 for i, entry c for NN[i, c], 0 where
    NN[i, c] = -1) of the sparse inverse factor of the Vecchia density."""
    locs = np.asarray(locs, dtype=np.float64)
    NN = np.asarray(NN)
    n, W = NN.shape
    theta = np.asarray(theta, dtype=np.float64)
    assert len(theta) == nparms(covfun, locs.shape[1] if locs.ndim == 2 else 1)
    B = np.zeros((n, W))
    for i in range(n):
        nb = [int(j) for j in NN[i, 1:] if j >= 0]
        pts = np.vstack([locs[[i]], locs[nb]]) if nb else locs[[i]]
        S = _cov_matrix(covfun, theta, pts)
        if nb:
            w = np.linalg.solve(S[1:, 1:], S[1:, 0])
            v = S[0, 0] - S[0, 1:] @ w
        else:
            w = np.zeros(0)
            v = S[0, 0]
        B[i, 0] = 1.0 / np.sqrt(v)
        B[i, 1:1 + len(nb)] = -w / np.sqrt(v)
    return B


def simulate(locs, NN, theta, covfun, z):
    """The sequential draw driven by the standard normal variates z (length n)."""
    B = factor_rows(locs, NN, theta, covfun)
    NN = np.asarray(NN)
    n, W = NN.shape
    y = np.zeros(n)
    for i in range(n):
        s = 0.0
        for c in range(1, W):
            j = int(NN[i, c])
            if j >= 0:
                s += B[i, c] * y[j]
        y[i] = (z[i] - s) / B[i, 0]
    return y

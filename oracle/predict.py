"""Oracle for Vecchia prediction and the nearest-neighbour search used for it -- TEST
INFRASTRUCTURE (see ``oracle/__init__``).

Prediction at a target from its neighbour set N (the Gaussian process conditional):
    mean = x*' beta + k' Sigma_NN^-1 (y_N - X_N beta),   var = c - k' Sigma_NN^-1 k,
Sigma_NN with the nugget sigma2 tau2 on its diagonal, k the covariances of the target with
N, c = sigma2 (latent field) or sigma2 (1 + tau2) (a new observation).  Covariances from the
oracle's ``cov_pairs``; the solve is numpy FP64 (numpy.linalg.solve).

Nearest neighbours: the m smallest keys (d2, j) over all reference points, d2 summed
coordinate by coordinate with separate roundings (numpy element-wise, no fused
multiply-add), by a stable sort.
"""
from __future__ import annotations

import numpy as np

from . import cov_pairs


def _cov(covfun, theta, A, B, same=False):
    ia, ib = np.meshgrid(np.arange(len(A)), np.arange(len(B)), indexing="ij")
    s = (ia.ravel() == ib.ravel()).astype(np.int32) if same else np.zeros(ia.size, np.int32)
    C, _ = cov_pairs(covfun, theta, A[ia.ravel()], B[ib.ravel()], s)
    return C.reshape(len(A), len(B))


def predict(locs, y, X, beta, locs_pred, X_pred, NN_pred, theta, covfun, latent=True):
    locs = np.asarray(locs, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    sig2, tau2 = theta[0], theta[-1]
    r = np.asarray(y) - np.asarray(X) @ np.asarray(beta)
    npred = len(locs_pred)
    mean = np.empty(npred)
    var = np.empty(npred)
    for q in range(npred):
        nb = [int(j) for j in NN_pred[q] if j >= 0]
        c = sig2 if latent else sig2 * (1.0 + tau2)
        xb = float(np.asarray(X_pred[q]) @ np.asarray(beta))
        if not nb:
            mean[q], var[q] = xb, c
            continue
        S = _cov(covfun, theta, locs[nb], locs[nb], same=True)
        k = _cov(covfun, theta, locs[nb], np.asarray(locs_pred)[[q]])[:, 0]
        w = np.linalg.solve(S, k)
        mean[q] = xb + w @ r[nb]
        var[q] = c - w @ k
    return mean, var


def squared_lags(A, B):
    """d2 between every row of A and every row of B (len(A) x len(B))."""
    d2 = None
    for k in range(A.shape[1]):
        t = A[:, k][:, None] - B[:, k][None, :]
        d2 = t * t if d2 is None else d2 + t * t
    return d2


def nearest(locs_ref, locs_query, m):
    locs_ref = np.asarray(locs_ref, dtype=np.float64)
    locs_query = np.asarray(locs_query, dtype=np.float64)
    out = -np.ones((len(locs_query), m), dtype=np.int32)
    for q0 in range(0, len(locs_query), 256):
        d2 = squared_lags(locs_query[q0:q0 + 256], locs_ref)
        for a in range(d2.shape[0]):
            order = np.lexsort((np.arange(len(locs_ref)), d2[a]))[:m]
            out[q0 + a, :len(order)] = order
    return out

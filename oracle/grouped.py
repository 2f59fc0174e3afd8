"""Oracle for grouped (joint) conditioning -- TEST INFRASTRUCTURE (see ``oracle/__init__``).

Sec. 2.1 (and Sec. 5, as future work) mentions grouping: several observations share one
conditional, which means fewer likelihood terms and a sharper approximation.  The
definitions used here:

* groups are contiguous ranges B_b = [s_b, e_b) of the ordering;
* group b conditions on U_b = (union over i in B_b of i's NNarray neighbours) minus B_b.
  Every neighbour of i precedes i, so U_b lies before s_b and the product of the group
  conditionals p(y_B | y_U) is a valid joint density;
* group b's contribution to Algorithm 1's sums is that of p(y_B | y_U).  Since the joint
  density of U and B is p(y_U) p(y_B | y_U), every summed quantity of the conditional is
  the quantity of the dense Gaussian block on U + B minus that of the block on U:
      logdet |S|, y' S^-1 y, X' S^-1 X, y' S^-1 X,
      d/dtheta_j of each: tr(S^-1 dS_j), -(S^-1 y)' dS_j (S^-1 y), ...,
      Fisher information 1/2 tr(S^-1 dS_j S^-1 dS_l).
Dense FP64 numpy (Cholesky solves) on the covariances of the oracle's ``cov_pairs``; the
record has the layout of the C oracle's, so ``oracle.profile`` finishes it.
"""
from __future__ import annotations

import numpy as np

from . import cov_pairs, nparms, profile, stats_len


def group_blocks(NN, group_off):
    """Block index lists from an NNarray and contiguous groups: block b is U_b (ascending)
    followed by the members s_b .. e_b - 1.  Returns (block_off, block_idx, nmemb)."""
    NN = np.asarray(NN)
    group_off = np.asarray(group_off, dtype=np.int64)
    blocks, nm = [], []
    for b in range(len(group_off) - 1):
        s, e = int(group_off[b]), int(group_off[b + 1])
        cond = set()
        for i in range(s, e):
            cond.update(int(j) for j in NN[i, 1:] if j >= 0)
        cond -= set(range(s, e))
        blocks.append(sorted(cond) + list(range(s, e)))
        nm.append(e - s)
    off = np.zeros(len(blocks) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(bl) for bl in blocks])
    idx = np.array([j for bl in blocks for j in bl], dtype=np.int32)
    return off, idx, np.array(nm, dtype=np.int32)


def _dense(covfun, theta, pts):
    k = len(pts)
    ia, ib = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    same = (ia.ravel() == ib.ravel()).astype(np.int32)
    C, dC = cov_pairs(covfun, theta, pts[ia.ravel()], pts[ib.ravel()], same)
    return C.reshape(k, k), dC.T.reshape(-1, k, k)


def block_record(covfun, theta, locs, y, X, idx):
    """The summed quantities of the dense Gaussian block on the observations idx, in the
    C oracle's record layout (zeros for an empty block)."""
    p = X.shape[1]
    q = nparms(covfun, locs.shape[1])
    rec = np.zeros(stats_len(p, q))
    if len(idx) == 0:
        return rec
    S, dS = _dense(covfun, theta, locs[idx])
    Lc = np.linalg.cholesky(S)
    solve = lambda B: np.linalg.solve(Lc.T, np.linalg.solve(Lc, B))  # noqa: E731
    yy, XX = y[idx], X[idx]
    Siy, SiX = solve(yy), solve(XX)
    Si = solve(np.eye(len(idx)))
    o = 0
    rec[o] = 2.0 * np.sum(np.log(np.diag(Lc))); o += 1
    rec[o] = yy @ Siy; o += 1
    rec[o:o + p * p] = (XX.T @ SiX).ravel(); o += p * p
    rec[o:o + p] = XX.T @ Siy; o += p
    SidS = [Si @ dS[j] for j in range(q)]
    rec[o:o + q] = [np.trace(SidS[j]) for j in range(q)]; o += q
    rec[o:o + q] = [-(Siy @ dS[j] @ Siy) for j in range(q)]; o += q
    rec[o:o + q * p * p] = np.concatenate([-(SiX.T @ dS[j] @ SiX).ravel() for j in range(q)]); o += q * p * p
    rec[o:o + q * p] = np.concatenate([-(SiX.T @ dS[j] @ Siy) for j in range(q)]); o += q * p
    rec[o:o + q * q] = np.array([[0.5 * np.sum(SidS[j] * SidS[l].T) for l in range(q)]
                                 for j in range(q)]).ravel()
    return rec


def stats(locs, y, X, block_off, block_idx, nmemb, theta, covfun):
    """Summed record over the groups: for each block, the record of (U + B) minus that of U
    (U = the block's first len - nmemb indices)."""
    locs = np.asarray(locs, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    q = nparms(covfun, locs.shape[1])
    tot = np.zeros(stats_len(X.shape[1], q))
    for b in range(len(block_off) - 1):
        idx = np.asarray(block_idx[block_off[b]:block_off[b + 1]], dtype=np.int64)
        nu = len(idx) - int(nmemb[b])
        tot += block_record(covfun, theta, locs, y, X, idx)
        tot -= block_record(covfun, theta, locs, y, X, idx[:nu])
    return tot


def loglik_grad_info(locs, y, X, block_off, block_idx, nmemb, theta, covfun):
    """Profiled-beta grouped Vecchia loglikelihood, gradient, Fisher information, betahat."""
    X = np.asarray(X, dtype=np.float64)
    rec = stats(locs, y, X, block_off, block_idx, nmemb, theta, covfun)
    n = int(np.sum(nmemb))
    q = nparms(covfun, np.asarray(locs).shape[1])
    ll, g, info, beta = profile(rec, n, X.shape[1], q)
    return {"loglik": ll, "grad": g, "info": info, "betahat": beta}

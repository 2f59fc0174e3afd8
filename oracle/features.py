"""Oracle for the binned empirical semivariogram features -- TEST INFRASTRUCTURE (see
``oracle/__init__``).

The paper does not define these features; they are the input of the library's learned
starting point for Fisher scoring.  Definition, for one field y (n values) at locs:

  * pairs: every (i, NN[i, c]) with c >= 1 and NN[i, c] >= 0, then P random pairs
    (floor(r1 n / 2^32), floor(r2 n / 2^32)) from the caller's 32-bit words (r1, r2);
  * squared lag h2 = sum over coordinates, in order, of (s_ik - s_jk)^2 (FP64);
  * bin k when edges2[k] <= h2 < edges2[k + 1] (edges2 ascending, nbins + 1 values);
    other pairs are ignored;
  * bin value = mean over its pairs of (y_i - y_j)^2 / 2, divided by the population
    variance of y; an empty bin copies the nearest non-empty bin (the lower one on a
    tie); with every bin empty the values are NaN.

numpy FP64 throughout; the feature vector is returned in FP64 (the library stores FP32).
"""
from __future__ import annotations

import numpy as np


def pair_indices(NN, n, rand_pairs):
    """(i, j) of every pair, NNarray pairs first, then the random ones."""
    NN = np.asarray(NN)
    m = NN.shape[1] - 1
    i_nn = np.repeat(np.arange(n), m)
    j_nn = NN[:, 1:].reshape(-1).astype(np.int64)
    keep = j_nn >= 0
    r = np.asarray(rand_pairs, dtype=np.uint64).reshape(-1, 2)
    i_r = ((r[:, 0] * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
    j_r = ((r[:, 1] * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
    return (np.concatenate([i_nn[keep], i_r]), np.concatenate([j_nn[keep], j_r]))


def squared_lags(locs, i, j):
    locs = np.asarray(locs, dtype=np.float64)
    h2 = None
    for k in range(locs.shape[1]):
        dk = locs[i, k] - locs[j, k]
        h2 = dk * dk if h2 is None else h2 + dk * dk
    return h2


def features(locs, NN, y, rand_pairs, edges2):
    """Returns (features (nbins,), bin sums, bin counts)."""
    y = np.asarray(y, dtype=np.float64)
    edges2 = np.asarray(edges2, dtype=np.float64)
    nbins = len(edges2) - 1
    i, j = pair_indices(NN, len(y), rand_pairs)
    h2 = squared_lags(locs, i, j)
    k = np.searchsorted(edges2, h2, side="right") - 1
    ok = (k >= 0) & (k < nbins)
    dy = y[i[ok]] - y[j[ok]]
    sums = np.bincount(k[ok], weights=0.5 * (dy * dy), minlength=nbins)
    counts = np.bincount(k[ok], minlength=nbins).astype(np.int64)
    var = np.var(y)
    vals = np.full(nbins, np.nan)
    for b in range(nbins):
        src = -1
        if counts[b] > 0:
            src = b
        else:
            for dist in range(1, nbins):
                if b - dist >= 0 and counts[b - dist] > 0:
                    src = b - dist
                    break
                if b + dist < nbins and counts[b + dist] > 0:
                    src = b + dist
                    break
        if src >= 0:
            vals[b] = sums[src] / counts[src] / var
    return vals, sums, counts


def log_edges2(nbins=32, lo=0.005, hi=0.5):
    """Squared edges of nbins log-spaced lag bins on [lo, hi]."""
    return np.geomspace(lo, hi, nbins + 1) ** 2

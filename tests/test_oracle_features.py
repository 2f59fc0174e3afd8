"""Pins for the semivariogram-feature oracle: closed forms on hand-built inputs, the
index map of the random pairs, invariances, the empty-bin rule, and the white-noise and
exponential-covariance expectations of the empirical semivariogram."""
import numpy as np

import workloads
from oracle import features as of


def test_line_with_linear_field_closed_form():
    # points on a line with spacing delta, each conditioning on its predecessor, y = a i:
    # every NNarray pair has lag delta and (y_i - y_j)^2 / 2 = a^2 / 2; var(y) = a^2 (n^2 - 1) / 12
    n, delta, a = 50, 0.01, 3.0
    locs = np.column_stack([np.arange(n) * delta, np.zeros(n)])
    NN = np.column_stack([np.arange(n), np.arange(n) - 1]).astype(np.int32)
    y = a * np.arange(n)
    e2 = of.log_edges2()
    f, s, c = of.features(locs, NN, y, np.zeros((0, 2), np.uint32), e2)
    k = np.searchsorted(e2, delta * delta, side="right") - 1
    assert c[k] == n - 1 and c.sum() == n - 1
    assert np.isclose(s[k], (n - 1) * a * a / 2, rtol=1e-14)
    assert np.allclose(f, 6.0 / (n * n - 1), rtol=1e-13)   # every bin copies bin k


def test_random_pair_index_map():
    n = 1000
    r = np.array([[0, 2**32 - 1], [2**31, 2**31 - 1], [123456789, 4000000000]], dtype=np.uint32)
    i, j = of.pair_indices(np.zeros((n, 1), np.int32), n, r)
    assert list(i) == [0, 500, 123456789 * n // 2**32]
    assert list(j) == [n - 1, 499, 4000000000 * n // 2**32]


def test_empty_bin_rule():
    # only bins 3 and 7 receive pairs: 0..5 copy 3 (5 is a tie, the lower bin wins), 6..9 copy 7
    e2 = np.arange(11, dtype=np.float64) ** 2
    locs = np.array([[0.0, 0.0], [3.5, 0.0], [0.0, 7.5]])
    NN = np.array([[0, -1], [1, 0], [2, 0]], dtype=np.int32)
    y = np.array([0.0, 1.0, 3.0])
    f, s, c = of.features(locs, NN, y, np.zeros((0, 2), np.uint32), e2)
    assert list(np.nonzero(c)[0]) == [3, 7]
    var = np.var(y)
    v3, v7 = 0.5 / var, 4.5 / var
    assert np.allclose(f, [v3] * 6 + [v7] * 4, rtol=1e-15)


def test_scale_and_shift_invariance():
    rng = np.random.default_rng(0)
    L = rng.uniform(size=(400, 2))
    L = L[workloads.maxmin_order(L)]
    NN = workloads.ordered_nn(L, 10)
    y = rng.standard_normal(400)
    r = rng.integers(0, 2**32, size=(5000, 2), dtype=np.uint64).astype(np.uint32)
    e2 = of.log_edges2()
    f1, _, c1 = of.features(L, NN, y, r, e2)
    f2, _, c2 = of.features(L, NN, -2.5 * y + 7.0, r, e2)
    assert np.array_equal(c1, c2) and np.allclose(f1, f2, rtol=1e-12)


def test_white_noise_gives_one():
    # E[(y_i - y_j)^2 / 2] = var for independent values
    rng = np.random.default_rng(1)
    n = 20000
    L = rng.uniform(size=(n, 2))
    NN = np.column_stack([np.arange(n), -np.ones(n)]).astype(np.int32)
    y = rng.standard_normal(n)
    r = rng.integers(0, 2**32, size=(2**20, 2), dtype=np.uint64).astype(np.uint32)
    f, _, c = of.features(L, NN, y, r, of.log_edges2())
    big = c > 5000
    assert big.sum() > 10 and np.all(np.abs(f[big] - 1.0) < 0.08)


def test_exponential_field_expectation():
    # E[(y_i - y_j)^2 / 2] = sigma2 (1 + tau2 - exp(-h / rho)) at lag h > 0; the sample
    # variance is close to sigma2 (1 + tau2) when rho is much smaller than the domain
    w = workloads.make_field(6000, 0, [1.0, 0.03, 0.1], 20, p=1, seed=2, sim="sequential",
                             beta=np.array([0.0]), m_sim=30)
    rng = np.random.default_rng(3)
    r = rng.integers(0, 2**32, size=(2**20, 2), dtype=np.uint64).astype(np.uint32)
    e2 = of.log_edges2()
    f, _, c = of.features(w.locs, w.NN, w.y, r, e2)
    h = np.sqrt(e2[:-1] * e2[1:]) ** 0.5   # geometric bin centres (lags)
    expect = (1.1 - np.exp(-h / 0.03)) / 1.1
    big = c > 3000
    assert big.sum() > 10
    assert np.all(np.abs(f[big] - expect[big]) < 0.15 * expect[big] + 0.03)

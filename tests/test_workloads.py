"""Preprocessing pins: grid-accelerated maxmin ordering and ordered nearest neighbours
must equal their brute-force definitions (Sec. 2.1 ordering, Sec. 3 NNarray)."""
import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("n,d,seed", [(1, 2, 0), (2, 2, 0), (500, 2, 1), (800, 3, 2),
                                      (300, 1, 3)])
def test_maxmin_matches_brute_force(n, d, seed):
    x = np.random.default_rng(seed).uniform(size=(n, d))
    assert np.array_equal(workloads.maxmin_order(x), workloads.maxmin_order(x, brute=True))


def test_maxmin_ties_on_a_lattice():
    g = np.stack(np.meshgrid(np.arange(9.0), np.arange(7.0)), -1).reshape(-1, 2)
    assert np.array_equal(workloads.maxmin_order(g), workloads.maxmin_order(g, brute=True))


def test_maxmin_definition():
    x = np.random.default_rng(5).uniform(size=(200, 2))
    o = workloads.maxmin_order(x)
    assert sorted(o) == list(range(200))
    c = x.mean(0)
    assert o[0] == np.argmin(((x - c) ** 2).sum(1))
    y = x[o]
    for k in range(1, 200):
        dmin = np.min(((y[k:, None, :] - y[None, :k, :]) ** 2).sum(-1), axis=1)
        assert dmin[0] == dmin.max()


@pytest.mark.parametrize("n,d,m,seed", [(400, 2, 10, 1), (700, 2, 30, 2), (600, 3, 12, 3),
                                        (50, 2, 60, 4), (300, 1, 5, 5)])
def test_ordered_nn_matches_brute_force(n, d, m, seed):
    x = np.random.default_rng(seed).uniform(size=(n, d))
    x = x[workloads.maxmin_order(x)]
    a = workloads.ordered_nn(x, m)
    b = workloads.ordered_nn(x, m, brute=True)
    assert np.array_equal(a, b)
    for i in range(n):
        assert a[i, 0] == i
        k = min(i, m)
        assert np.all(a[i, 1:1 + k] < i) and np.all(a[i, 1:1 + k] >= 0)
        assert np.all(a[i, 1 + k:] == -1)


def test_ordered_nn_on_clustered_points():
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.normal(0, 0.01, (300, 2)), rng.normal(5, 1.0, (300, 2))])
    x = x[workloads.maxmin_order(x)]
    assert np.array_equal(workloads.ordered_nn(x, 15), workloads.ordered_nn(x, 15, brute=True))


def test_small_exp_workload_shape():
    w = workloads.cfg_small_exp()
    assert w.n == 2000 and w.m == 10 and w.NN.shape == (2000, 11) and w.p == 1
    assert np.all(w.NN[:, 0] == np.arange(2000))


def test_batch_workload_layout_and_determinism():
    a = workloads.cfg_batch(seed=5, nbatch=7, n_range=(100, 600), m_choices=(0, 3, 8), m_sim=8)
    b = workloads.cfg_batch(seed=5, nbatch=7, n_range=(100, 600), m_choices=(0, 3, 8), m_sim=8)
    for k in ("locs", "y", "X", "NN", "offsets", "m", "theta_true", "theta_start"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    off = a.offsets
    assert off[0] == 0 and np.all(np.diff(off) >= 1) and off[-1] == len(a.y) == len(a.locs)
    assert a.NN.size == int(np.sum(np.diff(off) * (a.m.astype(np.int64) + 1)))
    for k in range(a.nbatch):
        w = a.dataset(k)
        n = w.n
        assert np.array_equal(w.NN[:, 0], np.arange(n))
        nb = w.NN[:, 1:]
        assert np.all((nb == -1) | ((nb >= 0) & (nb < np.arange(n)[:, None])))
        assert np.isclose(w.theta_start[0], np.var(w.y))

"""Pins for the prediction oracle: with every observation as a neighbour it is exact GP
prediction, checked against scikit-learn's Gaussian process regressor (an independent
implementation of the posterior); interpolation at an observed site as the nugget vanishes;
the new-observation variance exceeds the latent one by the nugget; the neighbour search
against scipy's k-d tree."""
import numpy as np
import pytest

import oracle
from oracle import predict as op


def _data(n, seed, d=2):
    rng = np.random.default_rng(seed)
    L = rng.uniform(size=(n, d))
    y = rng.standard_normal(n)
    X = np.column_stack([np.ones(n), L[:, 0]])
    return rng, L, y, X


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_all_neighbours_equals_exact_gp_posterior(nu):
    sk = pytest.importorskip("sklearn.gaussian_process")
    kern = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng, L, y, X = _data(120, 1)
    beta = np.array([0.3, -0.7])
    theta = np.array([1.4, 0.15, nu, 0.08])
    Lp = rng.uniform(size=(25, 2))
    Xp = np.column_stack([np.ones(25), Lp[:, 0]])
    NN = np.tile(np.arange(120, dtype=np.int32), (25, 1))
    mean, var = op.predict(L, y, X, beta, Lp, Xp, NN, theta, oracle.MATERN_ISO, latent=True)
    k = kern.ConstantKernel(theta[0], "fixed") * kern.Matern(
        length_scale=theta[1] * np.sqrt(2 * nu), length_scale_bounds="fixed", nu=nu)
    gp = sk.GaussianProcessRegressor(kernel=k, alpha=theta[0] * theta[3], optimizer=None,
                                     normalize_y=False)
    gp.fit(L, y - X @ beta)
    m_ref, s_ref = gp.predict(Lp, return_std=True)
    assert np.allclose(mean, Xp @ beta + m_ref, rtol=1e-8, atol=1e-10)
    assert np.allclose(var, s_ref ** 2, rtol=1e-7, atol=1e-12)


def test_interpolation_and_nugget_relation():
    rng, L, y, X = _data(60, 2)
    beta = np.array([0.5, 1.0])
    Lp = L[:5] + 0.0                      # targets at observed sites
    Xp = X[:5]
    NN = op.nearest(L, Lp, 12)
    th_small = np.array([1.0, 0.2, 1.5, 1e-10])
    mean, var = op.predict(L, y, X, beta, Lp, Xp, NN, th_small, oracle.MATERN_ISO, latent=True)
    assert np.allclose(mean, y[:5], atol=1e-6) and np.all(var < 1e-6)
    th = np.array([1.0, 0.2, 1.5, 0.1])
    _, vl = op.predict(L, y, X, beta, Lp, Xp, NN, th, oracle.MATERN_ISO, latent=True)
    _, vo = op.predict(L, y, X, beta, Lp, Xp, NN, th, oracle.MATERN_ISO, latent=False)
    assert np.allclose(vo - vl, th[0] * th[3], rtol=1e-12)


def test_nearest_against_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(3)
    ref = rng.uniform(size=(3000, 2))
    qry = rng.uniform(-0.1, 1.1, size=(400, 2))
    NN = op.nearest(ref, qry, 15)
    dist, idx = spatial.cKDTree(ref).query(qry, k=15)
    assert np.array_equal(NN, idx.astype(np.int32))
    NN3 = op.nearest(ref[:10], qry[:5], 15)           # fewer references than m
    assert np.all(NN3[:, 10:] == -1) and np.all(NN3[:, :10] >= 0)

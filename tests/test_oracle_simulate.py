"""Pins for the oracle's sequential Vecchia draw (Sec. 2.1, Eq. 3).

  * conditioning on every earlier point (m = n - 1) makes the Vecchia density exact, so
    the draw must equal L z with L the lower Cholesky factor of the dense covariance;
  * the factor rows must reproduce the Gaussian conditional law: the first row of the
    inverse of the block covariance (i first, then N(i)) is b_i0 * b_i, so its (0, 0)
    entry is 1/Var(y_i | y_N) = b_i0^2;
  * the diagonal entries give the Vecchia log determinant that the pass (Algorithm 1)
    accumulates: sum_i 2 log(1 / b_i0)."""
import numpy as np

import oracle
import workloads
from oracle import simulate as osim

EXP, MAT = oracle.EXP_ISO, oracle.MATERN_ISO


def _pts(n, seed):
    L = np.random.default_rng(seed).uniform(size=(n, 2))
    return L[workloads.maxmin_order(L)]


def test_full_conditioning_equals_dense_cholesky():
    n = 40
    locs = _pts(n, 1)
    NN = workloads.ordered_nn(locs, n - 1)
    z = np.random.default_rng(2).standard_normal(n)
    for covfun, th in ((EXP, [1.3, 0.2, 0.05]), (MAT, [0.8, 0.15, 1.3, 0.02])):
        y = osim.simulate(locs, NN, th, covfun, z)
        S = osim._cov_matrix(covfun, np.array(th), locs)
        assert np.allclose(y, np.linalg.cholesky(S) @ z, rtol=1e-10, atol=1e-11)


def test_factor_rows_are_the_conditional_law():
    n, m = 60, 6
    locs = _pts(n, 3)
    NN = workloads.ordered_nn(locs, m)
    th = np.array([1.1, 0.12, 0.9, 0.03])
    B = osim.factor_rows(locs, NN, th, MAT)
    for i in (0, 1, 5, 30, 59):
        nb = [int(j) for j in NN[i, 1:] if j >= 0]
        S = osim._cov_matrix(MAT, th, np.vstack([locs[[i]], locs[nb]]))
        P = np.linalg.inv(S)   # the (0, 0) entry of the block precision is 1 / Var(y_i | y_N)
        assert np.isclose(B[i, 0] ** 2, P[0, 0], rtol=1e-10)
        # the precision's first row is b_0 * b: P[0, c] = b_i0 * b_ic
        assert np.allclose(B[i, 1:1 + len(nb)] * B[i, 0], P[0, 1:], rtol=1e-9, atol=1e-12)


def test_factor_rows_give_the_pass_log_determinant():
    # sum_i 2 log(1 / b_i0) is the Vecchia log determinant the pass accumulates
    w = workloads.make_field(150, MAT, [1.0, 0.1, 1.5, 0.05], 8, p=1, seed=4, sim="sequential",
                             beta=np.array([0.0]), m_sim=12)
    B = osim.factor_rows(w.locs, w.NN, w.theta_true, MAT)
    rec, _ = oracle.stats(w.locs, w.y, w.X, w.NN, w.theta_true, MAT)
    parts = oracle.split_stats(rec, 1, 4)
    assert np.isclose(np.sum(-2.0 * np.log(B[:, 0])), parts["logdet"], rtol=1e-12)

"""Pins for the oracle's Vecchia pass (Algorithm 1 + the profile step of Sec. 3).

Independent references, all computed here with numpy/scipy dense linear algebra:
  * m = n-1: Vecchia is the exact Gaussian likelihood (Sec. 2.1), so loglik, gradient and
    Fisher information equal Eq. 1-2 evaluated densely (with 1/2, see the readings).
  * m < n: the Vecchia conditionals define a valid joint density with sparse inverse
    Cholesky factor (Sec. 2.1).  It is built densely from the conditional regressions
    and its loglik, GLS beta and finite-difference gradient are compared.
  * Per-observation Fisher information equals I(block) - I(neighbours) with
    I = 1/2 tr(S^-1 dS_j S^-1 dS_l), evaluated from dense inverses.
  * m = 0 closed forms.
Covariance matrices come from oracle.cov_pairs, which is pinned on its own in
test_oracle_covariance.py.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import workloads

EXP, MAT, ST = oracle.EXP_ISO, oracle.MATERN_ISO, oracle.EXP_SPACETIME
ANI = oracle.EXP_ANISO


def dense_cov(covfun, theta, locs):
    n, d = locs.shape
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    C, dC = oracle.cov_pairs(covfun, theta, locs[ii], locs[jj], (ii == jj).astype(np.int32))
    q = dC.shape[1]
    return C.reshape(n, n), dC.T.reshape(q, n, n)


def dense_gp(covfun, theta, locs, y, X):
    """Exact GP: loglik (Eq. 1 with 1/2), score (Eq. 2 with 1/2), Fisher info, GLS beta."""
    S, dS = dense_cov(covfun, theta, locs)
    cf = sla.cho_factor(S, lower=True)
    SiX = sla.cho_solve(cf, X)
    Siy = sla.cho_solve(cf, y)
    beta = np.linalg.solve(X.T @ SiX, X.T @ Siy)
    r = y - X @ beta
    Sir = sla.cho_solve(cf, r)
    logdet = 2 * np.sum(np.log(np.diag(cf[0])))
    n = len(y)
    ll = -0.5 * n * np.log(2 * np.pi) - 0.5 * logdet - 0.5 * r @ Sir
    q = dS.shape[0]
    SidS = [sla.cho_solve(cf, dS[j]) for j in range(q)]
    grad = np.array([-0.5 * np.trace(SidS[j]) + 0.5 * Sir @ dS[j] @ Sir for j in range(q)])
    info = np.array([[0.5 * np.sum(SidS[j] * SidS[l].T) for l in range(q)] for j in range(q)])
    return ll, grad, info, beta


def implied_loglik(covfun, theta, locs, y, X, NN):
    """Dense loglik of the joint density implied by the Vecchia conditionals."""
    n = len(y)
    S, _ = dense_cov(covfun, theta, locs)
    B = np.eye(n)
    dvec = np.empty(n)
    for i in range(n):
        nb = NN[i, 1:]
        nb = nb[nb >= 0]
        if len(nb):
            w = np.linalg.solve(S[np.ix_(nb, nb)], S[nb, i])
            B[i, nb] = -w
            dvec[i] = S[i, i] - S[i, nb] @ w
        else:
            dvec[i] = S[i, i]
    Q = B.T @ np.diag(1 / dvec) @ B
    beta = np.linalg.solve(X.T @ Q @ X, X.T @ Q @ y)
    r = y - X @ beta
    ll = -0.5 * n * np.log(2 * np.pi) - 0.5 * np.sum(np.log(dvec)) - 0.5 * r @ Q @ r
    return ll, beta


def small_case(covfun, n, m, p, seed, theta):
    return workloads.make_field(n, covfun, theta, m, p=p, seed=seed, sim="dense",
                                beta=np.linspace(0.5, -0.5, p))


CASES = [
    (EXP, [1.3, 0.15, 0.05], 1),
    (EXP, [0.7, 0.4, 0.2], 3),
    (MAT, [1.1, 0.1, 0.8, 0.03], 2),
    (MAT, [2.0, 0.05, 1.5, 0.05], 3),
    (MAT, [1.0, 0.2, 2.7, 0.01], 1),
    (ST, [1.0, 0.3, 0.5, 0.1], 2),
    (ANI, [1.2, 0.3, 0.6, 1.0, 0.05], 1),
    (ANI, [1.0, 0.2, 0.4, 0.6, 0.8, 1.0, 1.5, 0.1], 2),
]


def rel(a, b):
    return np.linalg.norm(np.atleast_1d(a - b)) / max(np.linalg.norm(np.atleast_1d(b)), 1e-300)


@pytest.mark.parametrize("covfun,theta,p", CASES)
def test_dense_exactness_m_equals_n_minus_1(covfun, theta, p):
    n = 60
    w = small_case(covfun, n, n - 1, p, seed=11, theta=theta)
    th = np.array(theta)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, covfun)
    ll, grad, info, beta = dense_gp(covfun, th, w.locs, w.y, w.X)
    assert abs(o["loglik"] - ll) <= 1e-11 * abs(ll)
    scale = max(np.linalg.norm(grad), np.sqrt(np.trace(info)))
    assert np.linalg.norm(o["grad"] - grad) <= 1e-10 * scale
    assert rel(o["info"], info) <= 1e-10
    assert np.linalg.norm(o["betahat"] - beta) <= 1e-10 * (np.linalg.norm(beta) + 1)


@pytest.mark.parametrize("covfun,theta,p", CASES)
def test_implied_density_and_gls_beta(covfun, theta, p):
    n, m = 36, 5
    w = small_case(covfun, n, m, p, seed=5, theta=theta)
    th = np.array(theta)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, covfun)
    ll, beta = implied_loglik(covfun, th, w.locs, w.y, w.X, w.NN)
    assert abs(o["loglik"] - ll) <= 1e-11 * abs(ll)
    assert np.linalg.norm(o["betahat"] - beta) <= 1e-10 * (np.linalg.norm(beta) + 1)


@pytest.mark.parametrize("covfun,theta,p", CASES)
def test_gradient_matches_finite_differences_of_implied_density(covfun, theta, p):
    n, m = 36, 5
    w = small_case(covfun, n, m, p, seed=9, theta=theta)
    th = np.array(theta)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, covfun)
    fd = np.empty(len(th))
    for j in range(len(th)):
        h = 1e-5 * th[j]
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd[j] = (implied_loglik(covfun, tp, w.locs, w.y, w.X, w.NN)[0]
                 - implied_loglik(covfun, tm, w.locs, w.y, w.X, w.NN)[0]) / (2 * h)
    scale = max(np.linalg.norm(fd), np.sqrt(np.trace(o["info"])))
    assert np.linalg.norm(o["grad"] - fd) <= 1e-6 * scale


@pytest.mark.parametrize("covfun,theta,p", CASES[:4] + CASES[-2:])
def test_per_point_info_is_block_minus_neighbour_information(covfun, theta, p):
    n, m = 25, 6
    w = small_case(covfun, n, m, p, seed=3, theta=theta)
    th = np.array(theta)
    recs = oracle.records(w.locs, w.y, w.X, w.NN, th, covfun)
    q = len(th)
    parts = oracle.split_stats(recs, p, q)
    S, dS = dense_cov(covfun, th, w.locs)

    def finfo(idx):
        if len(idx) == 0:
            return np.zeros((q, q))
        Si = np.linalg.inv(S[np.ix_(idx, idx)])
        A = [Si @ dS[j][np.ix_(idx, idx)] for j in range(q)]
        return np.array([[0.5 * np.sum(A[j] * A[l].T) for l in range(q)] for j in range(q)])

    for i in [0, 1, 4, 7, 12, 24]:
        nb = w.NN[i, 1:]
        nb = list(nb[nb >= 0])
        ref = finfo(nb + [i]) - finfo(nb)
        assert np.allclose(parts["ainfo"][i], ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_m_zero_closed_form():
    th = np.array([1.7, 0.2, 0.3])
    w = small_case(EXP, 40, 0, 2, seed=2, theta=th)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, EXP)
    v = th[0] * (1 + th[2])
    beta = np.linalg.lstsq(w.X, w.y, rcond=None)[0]
    r = w.y - w.X @ beta
    n = len(w.y)
    ll = -0.5 * n * np.log(2 * np.pi * v) - 0.5 * r @ r / v
    assert abs(o["loglik"] - ll) <= 1e-13 * abs(ll)
    dv = np.array([1 + th[2], 0.0, th[0]])  # dv/dsigma2, dv/drho, dv/dtau2
    info = 0.5 * n * np.outer(dv, dv) / v ** 2
    assert np.allclose(o["info"], info, rtol=1e-13, atol=1e-12)
    grad = -0.5 * dv * (n / v - r @ r / v ** 2)
    assert np.allclose(o["grad"], grad, rtol=1e-12, atol=1e-10)


def test_neighbour_order_within_a_row_does_not_matter():
    th = np.array([1.1, 0.1, 0.8, 0.03])
    w = small_case(MAT, 80, 8, 2, seed=21, theta=th)
    NN2 = w.NN.copy()
    rng = np.random.default_rng(0)
    for i in range(len(NN2)):
        k = int((NN2[i, 1:] >= 0).sum())
        NN2[i, 1:1 + k] = NN2[i, 1 + rng.permutation(k)]
    a = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, MAT)
    b = oracle.loglik_grad_info(w.locs, w.y, w.X, NN2, th, MAT)
    assert abs(a["loglik"] - b["loglik"]) <= 1e-12 * abs(a["loglik"])
    assert np.allclose(a["grad"], b["grad"], rtol=1e-10, atol=1e-9)
    assert np.allclose(a["info"], b["info"], rtol=1e-11)


def test_thread_count_does_not_change_result():
    th = np.array([1.0, 0.1, 0.02])
    w = small_case(EXP, 3000, 10, 1, seed=4, theta=th)
    s1, _ = oracle.stats(w.locs, w.y, w.X, w.NN, th, EXP, nthreads=1)
    s4, _ = oracle.stats(w.locs, w.y, w.X, w.NN, th, EXP, nthreads=4)
    assert np.array_equal(s1, s4)


def test_not_positive_definite_reports_first_bad_index():
    # two coincident points and an essentially zero nugget make the block singular
    th = np.array([1.0, 1.0, 20.0, 1e-300])
    w = small_case(MAT, 30, 4, 1, seed=1, theta=[1.0, 0.1, 1.5, 0.1])
    locs = w.locs.copy()
    j = int(w.NN[17, 1])
    locs[17] = locs[j]
    with pytest.raises(oracle.OracleError) as e:
        oracle.loglik_grad_info(locs, w.y, w.X, w.NN, th, MAT)
    assert e.value.code == 2
    assert 0 <= e.value.bad_index <= 17


def test_bad_nnarray_rejected():
    th = np.array([1.0, 0.1, 0.02])
    w = small_case(EXP, 20, 3, 1, seed=1, theta=th)
    NN = w.NN.copy()
    NN[10, 1] = 15  # a neighbour that is not earlier
    with pytest.raises(oracle.OracleError):
        oracle.loglik_grad_info(w.locs, w.y, w.X, NN, th, EXP)
    NN = w.NN.copy()
    NN[10, 0] = 9  # column 0 must be the observation itself
    with pytest.raises(oracle.OracleError):
        oracle.loglik_grad_info(w.locs, w.y, w.X, NN, th, EXP)

"""Pins for the oracle's Fisher scoring (Eq. 4) on log-parameters.

The optimum is checked against scipy.optimize (a different optimiser on the same
objective) and against the first-order condition g ~ 0."""
import numpy as np
import pytest
import scipy.optimize as so

import oracle
import workloads

EXP, MAT, ANI = oracle.EXP_ISO, oracle.MATERN_ISO, oracle.EXP_ANISO


@pytest.mark.parametrize("covfun,theta,start", [
    (EXP, [1.0, 0.1, 0.05], [0.5, 0.3, 0.2]),
    (MAT, [1.5, 0.08, 1.2, 0.05], [1.0, 0.15, 1.0, 0.1]),
    (ANI, [1.0, 0.1, 0.3, 0.8, 0.05], [0.6, 0.2, 0.2, 0.2, 0.2]),
])
def test_fisher_scoring_reaches_the_optimum(covfun, theta, start):
    w = workloads.make_field(500, covfun, theta, 10, p=2, seed=17, sim="dense",
                             beta=[1.0, -0.5])
    fit = oracle.fisher_fit(w.locs, w.y, w.X, w.NN, covfun, np.array(start), tol=1e-8)
    assert fit["status"] == 0
    assert 1 <= fit["iters"] <= 40
    # first-order condition on the log scale
    gt = fit["theta"] * fit["grad"]
    It = fit["theta"][:, None] * fit["info"] * fit["theta"][None, :]
    assert gt @ np.linalg.solve(It, gt) < 1e-8

    def negll(lt):
        try:
            return -oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, np.exp(lt), covfun)["loglik"]
        except oracle.OracleError:
            return np.inf

    def neggrad(lt):
        r = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, np.exp(lt), covfun)
        return -r["grad"] * np.exp(lt)

    res = so.minimize(negll, np.log(start), jac=neggrad, method="BFGS",
                      options={"gtol": 1e-9, "maxiter": 500})
    assert abs(-res.fun - fit["loglik"]) <= 1e-9 * abs(fit["loglik"])
    assert fit["loglik"] >= -res.fun - 1e-9 * abs(fit["loglik"])


def test_fit_trial_outside_domain_is_a_failed_trial():
    # a field whose likelihood rises towards the boundary (smoothness at its lower clamp,
    # nugget -> 0): late trials underflow the nugget to exactly 0, which must count as a
    # failed trial (step halved), so the fit ends with "no ascent" instead of an error
    bw = workloads.cfg_batch(seed=31, nbatch=6, n_range=(300, 1500), m_choices=(5, 10, 20),
                             m_sim=20)
    w = bw.dataset(5)
    fit = oracle.fisher_fit(w.locs, w.y, w.X, w.NN, w.covfun, w.theta_start)
    assert fit["status"] == 2
    assert fit["theta"][2] == 0.05 and fit["theta"][3] < 0.01
    start = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, w.theta_start, w.covfun)
    assert fit["loglik"] > start["loglik"]

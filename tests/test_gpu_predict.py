"""Vecchia prediction on the device against the oracle (FP64: mean and variance to 1e-10
relative) for the three covariance families, several m (0 to 80), latent and new-observation
variances; the query-point neighbour search bit-exact against the oracle's; errors."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import predict as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402

EXP, MAT, ST = vg.EXP_ISO, vg.MATERN_ISO, vg.EXP_SPACETIME


def _dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")


@pytest.mark.parametrize("nref,nq,d,m,seed", [(5000, 700, 2, 30, 1), (20000, 300, 2, 10, 2),
                                              (3000, 200, 3, 20, 3), (40, 50, 2, 60, 4),
                                              (8000, 500, 1, 12, 5)])
def test_nearest_matches_oracle(nref, nq, d, m, seed):
    rng = np.random.default_rng(seed)
    ref = rng.uniform(size=(nref, d))
    qry = rng.uniform(-0.2, 1.2, size=(nq, d))        # some queries outside the data's box
    got = vg.vecchia_nearest(_dev(ref), _dev(qry), m).cpu().numpy()
    assert np.array_equal(got, op.nearest(ref, qry, m))


@pytest.mark.parametrize("covfun,theta,m,p,latent", [
    (MAT, [1.3, 0.08, 1.5, 0.05], 30, 3, True),
    (MAT, [0.7, 0.2, 0.6, 0.01], 10, 1, False),
    (MAT, [2.0, 0.05, 2.3, 0.1], 80, 2, True),
    (EXP, [1.0, 0.1, 0.02], 20, 1, True),
    (EXP, [1.5, 0.3, 0.2], 0, 1, False),
    (ST, [1.0, 0.3, 0.4, 0.1], 25, 2, True),
])
def test_predict_matches_oracle(covfun, theta, m, p, latent):
    rng = np.random.default_rng(7)
    n, npred = 3000, 400
    d = 3 if covfun == ST else 2
    L = rng.uniform(size=(n, d))
    Lp = rng.uniform(size=(npred, d))
    X = np.column_stack([np.ones(n)] + [L[:, k % d] for k in range(p - 1)])
    Xp = np.column_stack([np.ones(npred)] + [Lp[:, k % d] for k in range(p - 1)])
    beta = np.linspace(0.5, -0.5, p)
    y = X @ beta + rng.standard_normal(n)
    NN = op.nearest(L, Lp, m) if m > 0 else np.zeros((npred, 0), np.int32)
    th = np.array(theta)
    mean, var, st = vg.vecchia_predict(_dev(L), _dev(y), _dev(X), _dev(beta), _dev(Lp), _dev(Xp),
                                       _dev(NN, torch.int32), _dev(th), covfun, latent=latent)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    mo, vo = op.predict(L, y, X, beta, Lp, Xp, NN, th, covfun, latent=latent)
    assert np.allclose(mean.cpu().numpy(), mo, rtol=1e-10, atol=1e-10 * np.abs(mo).max())
    assert np.allclose(var.cpu().numpy(), vo, rtol=1e-10, atol=1e-12)


def test_predict_on_the_fitted_benchmark_field():
    # the n = 1e5 Matern field: neighbours from the device search, prediction at 20 000 sites
    w = workloads.cfg_matern_100k()
    rng = np.random.default_rng(8)
    Lp = rng.uniform(size=(20000, 2))
    Xp = np.column_stack([np.ones(20000), Lp])
    beta = np.array([1.0, 0.5, -0.5])
    NN = vg.vecchia_nearest(_dev(w.locs), _dev(Lp), 30)
    mean, var, st = vg.vecchia_predict(_dev(w.locs), _dev(w.y), _dev(w.X), _dev(beta), _dev(Lp),
                                       _dev(Xp), NN, _dev(w.theta_true), w.covfun)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    sel = rng.choice(20000, 300, replace=False)
    mo, vo = op.predict(w.locs, w.y, w.X, beta, Lp[sel], Xp[sel], NN.cpu().numpy()[sel],
                        w.theta_true, w.covfun)
    assert np.allclose(mean.cpu().numpy()[sel], mo, rtol=1e-10, atol=1e-10)
    assert np.allclose(var.cpu().numpy()[sel], vo, rtol=1e-10)


def test_predict_reports_errors():
    rng = np.random.default_rng(9)
    L, Lp = rng.uniform(size=(100, 2)), rng.uniform(size=(10, 2))
    X, Xp, y, beta = np.ones((100, 1)), np.ones((10, 1)), rng.standard_normal(100), np.zeros(1)
    NN = op.nearest(L, Lp, 5)
    NN[3, 2] = 100                                      # index out of range
    _, _, st = vg.vecchia_predict(_dev(L), _dev(y), _dev(X), _dev(beta), _dev(Lp), _dev(Xp),
                                  _dev(NN, torch.int32), _dev([1.0, 0.1, 0.1]), EXP)
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [1, 3]
    NN = op.nearest(L, Lp, 5)
    _, _, st = vg.vecchia_predict(_dev(L), _dev(y), _dev(X), _dev(beta), _dev(Lp), _dev(Xp),
                                  _dev(NN, torch.int32), _dev([1.0, -0.1, 0.1]), EXP)
    torch.cuda.synchronize()
    assert int(st[0]) == 1

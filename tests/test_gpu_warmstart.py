"""What the learned start gains: a network trained (by the library's kernels) on fields
that the plain method simulated and fitted starts Fisher scoring closer to the optimum on
held-out fields, so the fits take fewer passes and reach the same optimum as the fits from
the default start; the fallback keeps the default where the prediction is worse.

"The same optimum" is the plain method's converged optimum, loglik within 1e-6 relative
(the default start's fit is the reference).  A Matern likelihood can have more than one local
maximum, and then the start decides which one Fisher scoring reaches: a field whose two
fits converge to different logliks passes only if the FP64 oracle confirms that both end
points are local maxima (stationary in the Fisher metric, and lower on both sides along
every parameter, 5% away on the log scale), and the learned start's maximum is not the
lower one.  One kind of maximum lies on the boundary: a fit whose nugget goes towards 0
stops where the log-scale gradient in it vanishes, and is stationary in the other
parameters."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402
from paper_2407_02740_gb300 import warmstart as ws  # noqa: E402


def _geometry(n, m, seed):
    L = np.random.default_rng(seed).uniform(size=(n, 2))
    L = L[workloads.maxmin_order(L)]
    return ws.make_geometry(L, workloads.ordered_nn(L, m), seed=seed)


@pytest.fixture(scope="module")
def trained():
    g = _geometry(1024, 20, 11)
    X, T, stats = ws.build_training_set(g, 3000, seed=12, chunk=1500, log=None)
    assert stats["converged"] >= 0.8 * stats["fields"]
    P, norm, losses = ws.train(X, T, epochs=80, batch=128, lr=2e-3, log=None)
    return P, norm, losses, X, T


def test_training_reduces_the_loss(trained):
    P, norm, losses, X, T = trained
    assert losses["final"] < 0.5 * losses["initial"]
    # the fit of the training targets: predictions explain part of each target's variance
    pred = vg.vecchia_mlp_forward(P, norm, X)
    resid = ((pred - T) ** 2).mean(dim=0)
    assert torch.all(resid < 0.6 * T.var(dim=0, unbiased=False))


def _stationary(locs, y, X, NN, th):
    # the fit rule's convergence measure at th, from the FP64 oracle: g~' I~^-1 g~ on the
    # log scale, over the parameters off the boundary.  A nugget driven towards 0 (which
    # the log-scale parametrisation reaches only in the limit) has a log-scale gradient
    # and information of ~0: that end is a boundary maximum, stationary in the others.
    o = oracle.loglik_grad_info(locs, y, X, NN, th, oracle.MATERN_ISO)
    free = np.ones(4, dtype=bool)
    free[3] = th[3] > 1e-12
    gt = (th * o["grad"])[free]
    It = (th[:, None] * o["info"] * th[None, :])[np.ix_(free, free)]
    return float(gt @ np.linalg.solve(It, gt)), o["loglik"]


def test_learned_start_takes_fewer_passes_to_the_same_optimum(trained):
    P, norm, _, _, _ = trained
    g = _geometry(4096, 20, 13)
    res = ws.evaluate(g, P, norm, nfields=48, seed=14, log=print, detail=True)
    det = res["fields_detail"]
    assert res["learned"]["converged"] >= res["default"]["converged"]
    assert res["both_converged"] >= 0.8 * 48
    assert res["max_loglik_diff_same"] <= 1e-6
    locs, X, NN = (g.locs.cpu().numpy(), g.X.cpu().numpy(), g.NN.cpu().numpy())
    differing = np.nonzero(det["converged_both"] & ~det["same"])[0]
    for f in differing:
        y = det["Y"][f]
        ends = []
        for th in (det["theta_default"][f], det["theta_learned"][f]):
            crit, ll = _stationary(locs, y, X, NN, th)
            assert crit < 1e-3, (f, th, crit)          # the fits stop below tol = 1e-4
            for j in range(4):                         # lower on both sides: a maximum
                for sg in (-1.0, 1.0):
                    th2 = th.copy()
                    th2[j] *= np.exp(0.05 * sg)
                    th2[2] = min(max(th2[2], 0.05), 20.0)
                    o2 = oracle.loglik_grad_info(locs, y, X, NN, th2, oracle.MATERN_ISO)
                    assert o2["loglik"] < ll + 1e-9 * abs(ll), (f, th, j, sg)
            ends.append(ll)
        scale = max(abs(ends[0]), len(y))
        assert abs(ends[0] - ends[1]) > 1e-6 * scale             # two distinct maxima
        assert ends[1] >= ends[0], f                              # the learned one not lower
    assert res["learned"]["mean_passes"] < res["default"]["mean_passes"]
    assert res["learned"]["fallback_rate"] < 0.5


def test_fallback_keeps_the_default_where_the_prediction_is_worse(trained):
    P, norm, _, _, _ = trained
    g = _geometry(1500, 20, 15)
    Y, _ = ws.simulate_fields(g, ws.sample_priors(np.random.default_rng(16), 6), 17)
    d0 = ws.default_start(Y)
    # a network whose output layer predicts an absurd range (rho = e^30) loses to the default
    bad = P.clone()
    bad[-4:] = 0.0
    bad[-4 - 512:-4] = 0.0
    badnorm = norm.clone()
    badnorm[64:68] = torch.tensor([0.0, 30.0, 0.0, 0.0], device=norm.device)
    start, used, feats = vg.vecchia_fields_warm_start(bad, badnorm, g.locs, g.X, g.NN, Y,
                                                      g.rand_pairs, g.edges2, d0)
    assert torch.all(used == 0) and torch.equal(start, d0)
    start, used, feats = vg.vecchia_fields_warm_start(P, norm, g.locs, g.X, g.NN, Y, g.rand_pairs,
                                                      g.edges2, d0)
    ref = vg.vecchia_fields_variogram(g.locs, g.NN, Y, g.rand_pairs, g.edges2)
    assert torch.equal(feats, ref)
    th = ws.predict_theta(P, norm, feats, Y)
    keep = used.bool()
    assert torch.allclose(start[keep], th[keep], rtol=1e-6)

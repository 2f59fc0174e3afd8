"""The mixed-precision pass (FP32 block arithmetic, FP64 sums, profile and Fisher step)
against the FP64 oracle, and the mixed-then-FP64 fit against the FP64 fit.

Stated bounds (loglik relative, gradient relative to max(|g|, sqrt(tr info)), information
relative Frobenius, betahat relative to |beta|+1) for the workloads tested here; they are
the mixed path's documented accuracy."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402

BOUNDS = {"loglik": 1e-6, "grad": 2e-4, "info": 2e-5, "beta": 5e-6}


def errors(g, o):
    scale = max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))
    return {"loglik": abs(g["loglik"] - o["loglik"]) / abs(o["loglik"]),
            "grad": np.linalg.norm(g["grad"] - o["grad"]) / scale,
            "info": np.linalg.norm(g["info"] - o["info"]) / np.linalg.norm(o["info"]),
            "beta": np.linalg.norm(g["betahat"] - o["betahat"]) / (np.linalg.norm(o["betahat"]) + 1)}


def dev_inputs(w):
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    return (t(w.locs, torch.float64), t(w.y, torch.float64), t(w.X, torch.float64),
            t(w.NN, torch.int32))


def mixed_pass(w, th, lanes=0):
    h = vg.Handle(0)
    h.set_lanes(lanes)
    try:
        out, st = vg.vecchia_loglik_grad_info(*dev_inputs(w), torch.tensor(th, device="cuda:0"),
                                              w.covfun, prec="mixed", handle=h)
        torch.cuda.synchronize()
        r = vg.unpack(out, len(th), w.p)
        r["status"] = int(st[0])
    finally:
        h.close()
    return r


CASES = [
    (vg.EXP_ISO, [1.0, 0.1, 0.01], 1, 10),
    (vg.MATERN_ISO, [2.0, 0.05, 1.5, 0.05], 3, 30),
    (vg.MATERN_ISO, [1.2, 0.1, 0.7, 0.02], 1, 20),
    (vg.EXP_SPACETIME, [1.0, 0.3, 0.4, 0.1], 2, 30),
]


@pytest.mark.parametrize("covfun,theta,p,m", CASES)
def test_mixed_pass_within_stated_bounds(covfun, theta, p, m):
    w = workloads.make_field(2377, covfun, theta, m, p=p, seed=3, sim="sequential",
                             beta=np.linspace(1.0, -0.5, p), m_sim=min(m + 10, 60))
    th = np.array(theta)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, covfun)
    g = mixed_pass(w, th)
    assert g["status"] == 0
    err = errors(g, o)
    print("mixed errors", covfun, err)
    for k, b in BOUNDS.items():
        assert err[k] <= b, (k, err)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_mixed_every_lane_mapping(lanes):
    th = np.array([1.5, 0.07, 1.2, 0.05])
    w = workloads.make_field(900, vg.MATERN_ISO, th, 12, p=2, seed=5, sim="sequential",
                             beta=[1.0, -0.5], m_sim=20)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, vg.MATERN_ISO)
    try:
        g = mixed_pass(w, th, lanes=lanes)
    except vg.VecchiaError as e:
        assert e.code == 7
        return
    err = errors(g, o)
    for k, b in BOUNDS.items():
        assert err[k] <= b, (k, err)


def test_mixed_then_fp64_fit_reaches_the_fp64_optimum():
    th = [2.0, 0.05, 1.5, 0.05]
    w = workloads.make_field(4000, vg.MATERN_ISO, th, 20, p=3, seed=8, sim="sequential",
                             beta=[1.0, 0.5, -0.5], m_sim=30)
    args = dev_inputs(w)
    start = [float(np.var(w.y)), 0.1, 1.0, 0.1]
    h = vg.Handle(0)
    try:
        a = vg.vecchia_fit(*args, vg.MATERN_ISO, start, tol=1e-6, handle=h)
        b = vg.vecchia_fit(*args, vg.MATERN_ISO, start, tol=1e-6, prec="mixed", handle=h)
    finally:
        h.close()
    assert a["status"] == 0 and b["status"] == 0
    assert abs(a["loglik"] - b["loglik"]) <= 1e-8 * abs(a["loglik"])
    assert np.allclose(a["theta"], b["theta"], rtol=1e-4)


def _mixed_bounds(tau2):
    # the bands stated for the mixed path (FP64 pivots and per-observation dot products):
    # the tau2 >= 0.05 bounds above, a wider betahat bound down to 0.01, then wider bounds
    # down to 0.001 (measured worst cases there: loglik 2e-6, gradient 3.3e-4, information
    # 2.9e-5, betahat 6.9e-5)
    if tau2 >= 0.05:
        return BOUNDS
    if tau2 >= 0.01:
        return dict(BOUNDS, beta=5e-5)
    return {"loglik": 1e-5, "grad": 1e-3, "info": 1e-4, "beta": 2e-4}


@pytest.mark.parametrize("tau2", [0.05, 0.01, 0.003, 0.001])
@pytest.mark.parametrize("nu,rho,m", [(0.5, 0.1, 10), (1.5, 0.05, 20), (2.5, 0.2, 40),
                                      (1.5, 0.3, 30)])
def test_mixed_pass_small_nugget_bands(tau2, nu, rho, m):
    # nugget-dominated conditioning: the regime the FP64 pivots are for
    th = np.array([1.3, rho, nu, tau2])
    w = workloads.make_field(3000, vg.MATERN_ISO, th, m, p=1, seed=int(1000 * tau2) + m,
                             sim="sequential", beta=[0.5], m_sim=min(m + 10, 60))
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, vg.MATERN_ISO)
    g = mixed_pass(w, th)
    assert g["status"] == 0
    err = errors(g, o)
    err["loglik"] = abs(g["loglik"] - o["loglik"]) / max(abs(o["loglik"]), w.n)
    for k, b in _mixed_bounds(tau2).items():
        assert err[k] <= b, (k, tau2, err)

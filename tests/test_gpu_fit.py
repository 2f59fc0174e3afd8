"""Fisher scoring on the device (Eq. 4) against the oracle's Fisher scoring, which follows
the same rules: same optimum, same number of accepted steps."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402


def dev_inputs(w):
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    return (t(w.locs, torch.float64), t(w.y, torch.float64), t(w.X, torch.float64),
            t(w.NN, torch.int32))


@pytest.mark.parametrize("covfun,theta,start,p,m", [
    (vg.MATERN_ISO, [1.5, 0.08, 1.2, 0.05], [1.0, 0.15, 1.0, 0.1], 2, 15),
    (vg.EXP_ISO, [1.0, 0.1, 0.05], [0.5, 0.3, 0.2], 1, 10),
    (vg.EXP_SPACETIME, [1.0, 0.3, 0.5, 0.1], [0.7, 0.5, 0.3, 0.2], 2, 12),
])
def test_device_fit_matches_oracle_fit(covfun, theta, start, p, m):
    w = workloads.make_field(1500, covfun, theta, m, p=p, seed=31, sim="sequential",
                             beta=np.linspace(1.0, -0.5, p), m_sim=m + 5)
    o = oracle.fisher_fit(w.locs, w.y, w.X, w.NN, covfun, np.array(start), tol=1e-6)
    h = vg.Handle(0)
    try:
        g = vg.vecchia_fit(*dev_inputs(w), covfun, start, tol=1e-6, handle=h)
    finally:
        h.close()
    assert o["status"] == 0 and g["status"] == 0
    assert g["iters"] == o["iters"]
    assert abs(g["loglik"] - o["loglik"]) <= 1e-10 * abs(o["loglik"])
    assert np.allclose(g["theta"], o["theta"], rtol=1e-7, atol=0)
    assert np.allclose(g["betahat"], o["betahat"], rtol=1e-7, atol=1e-9)


def test_graph_and_host_loop_agree_bitwise():
    th = [1.2, 0.1, 0.8, 0.02]
    w = workloads.make_field(1200, vg.MATERN_ISO, th, 12, p=1, seed=3, sim="dense")
    args = dev_inputs(w)
    h = vg.Handle(0)
    try:
        a = vg.vecchia_fit(*args, vg.MATERN_ISO, [1.0, 0.2, 1.0, 0.1], tol=1e-8, handle=h)
        b = vg.vecchia_fit(*args, vg.MATERN_ISO, [1.0, 0.2, 1.0, 0.1], tol=1e-8, use_graph=False,
                           handle=h)
        c = vg.vecchia_fit(*args, vg.MATERN_ISO, [1.0, 0.2, 1.0, 0.1], tol=1e-8, handle=h)  # cached graph
    finally:
        h.close()
    for r in (b, c):
        assert np.array_equal(a["theta"], r["theta"]) and a["loglik"] == r["loglik"]
        assert a["iters"] == r["iters"] and a["evals"] == r["evals"]


def test_iteration_limit_and_bad_start():
    th = [1.0, 0.1, 0.05]
    w = workloads.make_field(400, vg.EXP_ISO, th, 8, p=1, seed=5, sim="dense")
    args = dev_inputs(w)
    r = vg.vecchia_fit(*args, vg.EXP_ISO, [0.3, 0.5, 0.3], maxit=0)
    assert r["status"] == 1 and r["iters"] == 0 and r["evals"] == 1
    assert np.allclose(r["theta"], [0.3, 0.5, 0.3])
    r2 = vg.vecchia_fit(*args, vg.EXP_ISO, [0.3, 0.5, 0.3], maxit=2)
    assert r2["iters"] <= 2 and r2["loglik"] >= r["loglik"]
    with pytest.raises(vg.VecchiaError):
        vg.vecchia_fit(*args, vg.EXP_ISO, [0.3, -0.5, 0.3])


def test_autotune_picks_a_mapping_and_round_trips(tmp_path):
    th = np.array([2.0, 0.05, 1.5, 0.05])
    w = workloads.make_field(3000, vg.MATERN_ISO, th, 30, p=3, seed=9, sim="sequential",
                             beta=[1.0, 0.5, -0.5], m_sim=35)
    args = dev_inputs(w)
    cp = torch.tensor(th, device="cuda:0")
    h = vg.Handle(0)
    try:
        r = vg.vecchia_autotune(*args, cp, vg.MATERN_ISO, handle=h)
        assert r["lanes"] in (1, 2, 4, 8, 16, 32) and r["threads"] in (64, 96, 128, 192, 256)
        assert r["ms"] > 0
        path = str(tmp_path / "tune.json")
        h.autotune_save(path)
        h2 = vg.Handle(0)
        h2.autotune_load(path)
        out, st = vg.vecchia_loglik_grad_info(*args, cp, vg.MATERN_ISO, handle=h2)
        torch.cuda.synchronize()
        g = vg.unpack(out, 4, 3)
        o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, vg.MATERN_ISO)
        assert int(st[0]) == 0
        assert abs(g["loglik"] - o["loglik"]) <= 1e-10 * abs(o["loglik"])
        h2.close()
    finally:
        h.close()

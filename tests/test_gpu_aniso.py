"""The exponential with one range per coordinate (Sec. 4.3, the Elevators form; q = d + 2)
on the device against the FP64 oracle, through the C ABI: covariance pairs, the FP64 pass
at every lane mapping (1e-10, the FP64 tolerance of the isotropic families), the full-size
Elevators-like workload, the mixed pass (the mixed path's stated bounds), the batched pass,
the device fit, prediction, and argument errors."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import predict as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402

ANI = vg.EXP_ANISO
TOL = 1e-10
MIXED_BOUNDS = {"loglik": 1e-6, "grad": 2e-4, "info": 2e-5, "beta": 5e-6}


def _dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=torch.device("cuda:0"))


def _errors(g, o, n):
    scale = max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))
    return {"loglik": abs(g["loglik"] - o["loglik"]) / max(abs(o["loglik"]), n),
            "grad": np.linalg.norm(g["grad"] - o["grad"]) / scale,
            "grad_j": float(np.max(np.abs(g["grad"] - o["grad"]) / np.maximum(
                np.sqrt(np.abs(np.diag(o["info"]))), 1e-4 * max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))))),
            "info": np.linalg.norm(g["info"] - o["info"]) / np.linalg.norm(o["info"]),
            "beta": np.linalg.norm(g["betahat"] - o["betahat"]) / (np.linalg.norm(o["betahat"]) + 1)}


def _pass(w, th, lanes=0, prec="fp64", threads=0):
    h = vg.Handle(0)
    h.set_lanes(lanes)
    h.set_block_threads(threads)
    try:
        out, st = vg.vecchia_loglik_grad_info(_dev(w.locs), _dev(w.y), _dev(w.X),
                                              _dev(w.NN, torch.int32), _dev(th), ANI, prec=prec,
                                              handle=h)
        torch.cuda.synchronize()
        r = vg.unpack(out, len(th), w.p)
        r["status"] = int(st[0])
    finally:
        h.close()
    return r


def _field(n, d, m, p, seed, tau2=0.1):
    rho = np.exp(np.linspace(np.log(0.15), np.log(1.5), d))
    th = np.concatenate([[1.3], rho, [tau2]])
    w = workloads.make_field(n, ANI, th, m, p=p, seed=seed, sim="sequential",
                             beta=np.linspace(1.0, -0.5, p), m_sim=min(m + 10, 40))
    return w, th


def test_covariance_pairs_match_oracle():
    rng = np.random.default_rng(1)
    for d in (1, 5, 18, 20):
        th = np.concatenate([[1.7], rng.uniform(0.1, 3.0, d), [0.04]])
        la = rng.uniform(-1, 1, size=(500, d))
        lb = la + rng.normal(0, 0.4, size=(500, d))
        lb[:3] = la[:3]                                   # coincident pairs
        same = np.zeros(500, np.int32)
        same[:2] = 1                                      # two diagonal entries
        C, dC = vg.vecchia_covariance_pairs(ANI, _dev(th), _dev(la), _dev(lb), _dev(same, torch.int32))
        Co, dCo = oracle.cov_pairs(ANI, th, la, lb, same)
        assert dC.shape == (500, d + 2)
        assert np.allclose(C.cpu().numpy(), Co, rtol=1e-14, atol=1e-300)
        assert np.allclose(dC.cpu().numpy(), dCo, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("n,d,m,p,seed", [(1500, 3, 10, 1, 1), (1200, 18, 30, 1, 2),
                                          (900, 6, 20, 2, 3), (400, 18, 60, 1, 4),
                                          (700, 1, 12, 2, 5), (500, 20, 0, 1, 6)])
def test_fp64_pass_matches_oracle(n, d, m, p, seed):
    w, th = _field(n, d, m, p, seed)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, ANI)
    lanes = [0, 4, 8, 16, 32] if (d, m) == (18, 30) else [0]
    for L in lanes:
        g = _pass(w, th, lanes=L)
        assert g["status"] == 0
        e = _errors(g, o, 0)
        assert max(e.values()) <= TOL, (L, e)


def test_full_size_elevators_like_workload():
    # n = 15000 attributes-as-locations, d = 18, m = 30 at the true and at the start values
    w = workloads.cfg_elevators_like()
    for th in (w.theta_true, w.theta_start):
        o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, ANI)
        g = _pass(w, th)
        assert g["status"] == 0
        e = _errors(g, o, 0)
        assert max(e.values()) <= TOL, e


def test_mixed_pass_within_stated_bounds():
    w, th = _field(2377, 8, 30, 1, seed=7)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, ANI)
    for L in (0, 8, 32):
        g = _pass(w, th, lanes=L, prec="mixed")
        assert g["status"] == 0
        e = _errors(g, o, 0)
        assert all(e[k] <= MIXED_BOUNDS[k] for k in MIXED_BOUNDS), (L, e)


def test_batched_pass_matches_oracle():
    fields = [_field(n, 5, m, 1, seed) for n, m, seed in
              ((800, 10, 11), (1300, 25, 12), (300, 0, 13), (2100, 30, 14), (50, 60, 15))]
    off = np.cumsum([0] + [w.n for w, _ in fields])
    locs = np.concatenate([w.locs for w, _ in fields])
    y = np.concatenate([w.y for w, _ in fields])
    X = np.concatenate([w.X for w, _ in fields])
    NN = np.concatenate([w.NN.reshape(-1) for w, _ in fields])
    th = np.stack([t * (1.0 + 0.1 * k) for k, (_, t) in enumerate(fields)])
    h = vg.Handle(0)
    try:
        out, st = vg.vecchia_batch_loglik_grad_info(
            _dev(locs), _dev(y), _dev(X), _dev(NN, torch.int32), list(off),
            [w.m for w, _ in fields], _dev(th), ANI, handle=h)
        torch.cuda.synchronize()
    finally:
        h.close()
    st = st.cpu().numpy()
    assert np.all(st[:, 0] == 0)
    for b, (w, _) in enumerate(fields):
        o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th[b], ANI)
        g = vg.unpack(out[b], th.shape[1], 1)
        e = _errors(g, o, 0)
        assert max(e.values()) <= TOL, (b, e)


def test_device_fit_matches_oracle_fit():
    w, th = _field(1500, 4, 15, 1, seed=21)
    start = np.concatenate([[1.0], np.full(4, 0.5), [0.2]])
    o = oracle.fisher_fit(w.locs, w.y, w.X, w.NN, ANI, start, tol=1e-6)
    h = vg.Handle(0)
    try:
        g = vg.vecchia_fit(_dev(w.locs), _dev(w.y), _dev(w.X), _dev(w.NN, torch.int32), ANI,
                           start, tol=1e-6, handle=h)
    finally:
        h.close()
    assert o["status"] == 0 and g["status"] == 0
    assert g["iters"] == o["iters"]
    assert abs(g["loglik"] - o["loglik"]) <= 1e-10 * abs(o["loglik"])
    assert np.allclose(g["theta"], o["theta"], rtol=1e-7, atol=0)


def test_prediction_matches_oracle():
    w, th = _field(3000, 6, 20, 2, seed=31)
    rng = np.random.default_rng(2)
    Lp = rng.uniform(size=(300, 6))
    Xp = np.column_stack([np.ones(300), Lp[:, 0]])
    beta = np.array([1.0, -0.5])
    NN = op.nearest(w.locs / th[1:-1], Lp / th[1:-1], 25)
    mean, var, st = vg.vecchia_predict(_dev(w.locs), _dev(w.y), _dev(w.X), _dev(beta), _dev(Lp),
                                       _dev(Xp), _dev(NN, torch.int32), _dev(th), ANI)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    mo, vo = op.predict(w.locs, w.y, w.X, beta, Lp, Xp, NN, th, ANI)
    assert np.allclose(mean.cpu().numpy(), mo, rtol=1e-10, atol=1e-10 * np.abs(mo).max())
    assert np.allclose(var.cpu().numpy(), vo, rtol=1e-10, atol=1e-12)


def test_argument_errors():
    w, th = _field(200, 4, 5, 1, seed=41)
    bad = th.copy()
    bad[3] = -0.2                                            # a negative range
    r = _pass(w, bad)
    assert r["status"] == 1 and np.isnan(r["loglik"])
    with pytest.raises(ValueError):                         # more than 20 coordinates
        vg.nparms(ANI, 21)
    assert vg.lib().vecchia_nparms_d(ANI, 21) == -1


def test_batched_fit_matches_oracle_fits():
    fields = [_field(n, 3, m, 1, seed) for n, m, seed in ((900, 12, 51), (1400, 15, 52))]
    off = np.cumsum([0] + [w.n for w, _ in fields])
    locs = np.concatenate([w.locs for w, _ in fields])
    y = np.concatenate([w.y for w, _ in fields])
    X = np.concatenate([w.X for w, _ in fields])
    NN = np.concatenate([w.NN.reshape(-1) for w, _ in fields])
    start = np.tile(np.concatenate([[1.0], np.full(3, 0.5), [0.2]]), (len(fields), 1))
    h = vg.Handle(0)
    try:
        r = vg.vecchia_batch_fit(_dev(locs), _dev(y), _dev(X), _dev(NN, torch.int32), list(off),
                                 [w.m for w, _ in fields], ANI, _dev(start), tol=1e-6, handle=h)
    finally:
        h.close()
    theta = r["theta"].cpu().numpy() if hasattr(r["theta"], "cpu") else np.asarray(r["theta"])
    for b, (w, _) in enumerate(fields):
        o = oracle.fisher_fit(w.locs, w.y, w.X, w.NN, ANI, start[b], tol=1e-6)
        assert o["status"] == 0 and int(r["status"][b]) == 0
        assert np.allclose(theta[b], o["theta"], rtol=1e-7, atol=0)

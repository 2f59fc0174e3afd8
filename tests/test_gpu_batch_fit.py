"""Batched Fisher scoring: every dataset of one batched fit follows the same path as its
own single-dataset device fit under the same kernel mapping (same statuses and step
counts, loglik to 1e-10 relative), reaches the oracle's optimum, and the CUDA-graph loop
equals the host-driven loop bit for bit; plus the batched autotuner."""
import json

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=torch.device("cuda:0"))


def _inputs(bw):
    return (_dev(bw.locs, torch.float64), _dev(bw.y, torch.float64), _dev(bw.X, torch.float64),
            _dev(bw.NN, torch.int32))


@pytest.fixture(scope="module")
def small_batch():
    return workloads.cfg_batch(seed=31, nbatch=6, n_range=(300, 1500), m_choices=(5, 10, 20),
                               m_sim=20)


def test_batch_fit_matches_single_fits(small_batch):
    bw = small_batch
    h = vg.Handle(0)
    h.set_lanes(8)
    h.set_block_threads(128)
    try:
        r = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun,
                                 _dev(bw.theta_start, torch.float64), handle=h)
        theta = r["theta"].cpu().numpy()
        out = r["out"].cpu().numpy()
        for b in range(bw.nbatch):
            w = bw.dataset(b)
            s = vg.vecchia_fit(_dev(w.locs, torch.float64), _dev(w.y, torch.float64),
                               _dev(w.X, torch.float64), _dev(w.NN, torch.int32), w.covfun,
                               w.theta_start, handle=h)
            assert r["status"][b] == s["status"]
            assert r["iters"][b] == s["iters"] and r["evals"][b] == s["evals"]
            assert abs(out[b, 0] - s["loglik"]) <= 1e-10 * abs(s["loglik"])
            np.testing.assert_allclose(theta[b], s["theta"], rtol=1e-7)
            g = vg.unpack(out[b], 4, 1)
            np.testing.assert_allclose(g["grad"], s["grad"], rtol=1e-6,
                                       atol=1e-6 * np.abs(s["grad"]).max() + 1e-9)
    finally:
        h.close()


def test_batch_fit_reaches_oracle_optimum(small_batch):
    bw = small_batch
    r = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun,
                             _dev(bw.theta_start, torch.float64))
    out = r["out"].cpu().numpy()
    assert np.sum(r["status"] == 0) >= bw.nbatch - 1
    for b in range(bw.nbatch):
        w = bw.dataset(b)
        o = oracle.fisher_fit(w.locs, w.y, w.X, w.NN, w.covfun, w.theta_start)
        # same rules, same path: same outcome and the same final loglik
        assert r["status"][b] == o["status"]
        assert abs(out[b, 0] - o["loglik"]) <= 1e-8 * abs(o["loglik"])


def test_batch_fit_graph_equals_host_loop(small_batch):
    bw = small_batch
    start = _dev(bw.theta_start, torch.float64)
    a = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun, start, use_graph=True)
    b = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun, start, use_graph=False)
    assert torch.equal(a["theta"], b["theta"]) and torch.equal(a["out"], b["out"])
    assert np.array_equal(a["iters"], b["iters"]) and np.array_equal(a["evals"], b["evals"])


def test_batch_fit_mixed_reaches_fp64_optimum(small_batch):
    bw = small_batch
    start = _dev(bw.theta_start, torch.float64)
    f64 = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun, start)
    mix = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun, start, prec="mixed")
    l64 = f64["out"][:, 0].cpu().numpy()
    lmx = mix["out"][:, 0].cpu().numpy()
    conv = f64["status"] == 0
    assert np.sum(conv) >= bw.nbatch - 1
    # where the FP64 fit converges, the mixed fit (FP64 phase last) converges to the same
    # optimum; elsewhere it ends the same way
    assert np.all(mix["status"][conv] == 0)
    assert np.all(mix["status"][~conv] == f64["status"][~conv])
    assert np.all(np.abs(lmx[conv] - l64[conv]) <= 1e-6 * np.abs(l64[conv]))


def test_batch_fit_bad_start_fails_only_that_dataset(small_batch):
    bw = small_batch
    st = bw.theta_start.copy()
    st[1, 2] = 25.0    # smoothness outside [0.05, 20]
    st[4, 0] = -1.0    # negative variance
    r = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun, _dev(st, torch.float64),
                             maxit=5)
    assert r["status"][1] == 3 and r["status"][4] == 3
    others = [b for b in range(bw.nbatch) if b not in (1, 4)]
    assert np.all(r["status"][others] != 3)
    assert np.all(np.isfinite(r["out"][others, 0].cpu().numpy()))


def test_batch_fit_maxit_zero_returns_start_values(small_batch):
    bw = small_batch
    start = _dev(bw.theta_start, torch.float64)
    r = vg.vecchia_batch_fit(*_inputs(bw), bw.offsets, bw.m, bw.covfun, start, maxit=0)
    assert np.all(r["iters"] == 0) and np.all(r["evals"] == 1)
    assert torch.equal(r["theta"], start)
    res, _ = vg.vecchia_batch_loglik_grad_info(*_inputs(bw), bw.offsets, bw.m, start, bw.covfun)
    torch.cuda.synchronize()
    assert torch.allclose(r["out"][:, 0], res[:, 0], rtol=1e-13, atol=0)


def test_batch_autotune_records_and_uses_mapping(tmp_path):
    # one block-size class (m + 1 <= 16): the tuned mapping is the plan's, and forcing it
    # gives the same kernels and tiles, hence bitwise equal results
    bw = workloads.cfg_batch(seed=32, nbatch=5, n_range=(500, 3000), m_choices=(8, 12),
                             m_sim=20)
    h = vg.Handle(0)
    try:
        cp = _dev(bw.theta_true, torch.float64)
        t = vg.vecchia_batch_autotune(*_inputs(bw), bw.offsets, bw.m, cp, bw.covfun, reps=2,
                                      handle=h)
        assert t["lanes"] in (1, 2, 4, 8, 16, 32) and t["threads"] in (64, 96, 128, 192, 256)
        path = str(tmp_path / "tune.json")
        h.autotune_save(path)
        txt = open(path).read()
        assert '"prec": 2' in txt
        auto, _ = vg.vecchia_batch_loglik_grad_info(*_inputs(bw), bw.offsets, bw.m, cp, bw.covfun,
                                                    handle=h)
        h2 = vg.Handle(0)
        h2.set_lanes(t["lanes"])
        h2.set_block_threads(t["threads"])
        forced, _ = vg.vecchia_batch_loglik_grad_info(*_inputs(bw), bw.offsets, bw.m, cp,
                                                      bw.covfun, handle=h2)
        torch.cuda.synchronize()
        h2.close()
        assert torch.equal(auto, forced)
    finally:
        h.close()


def test_batch_autotune_per_class(tmp_path):
    # datasets in two block-size classes (m = 10 and m = 20): one record per class, keyed by
    # the class's largest m, and a plan made afterwards uses each class's record
    bw = workloads.cfg_batch(seed=33, nbatch=6, n_range=(500, 3000), m_choices=(10, 20),
                             m_sim=20)
    h = vg.Handle(0)
    try:
        cp = _dev(bw.theta_true, torch.float64)
        vg.vecchia_batch_autotune(*_inputs(bw), bw.offsets, bw.m, cp, bw.covfun, reps=1, handle=h)
        path = str(tmp_path / "tune.json")
        h.autotune_save(path)
        recs = {r["m"]: r for r in json.load(open(path)) if r["prec"] == 2}
        assert set(recs) == {10, 20}
        plan = vg.BatchPlan(bw.offsets, bw.m, 2, 1, bw.covfun, handle=h)
        try:
            cls = plan.mapping()["classes"]
        finally:
            plan.close()
        assert [c["mmax"] for c in cls] == [10, 20]
        for c in cls:
            assert (c["lanes"], c["threads"]) == (recs[c["mmax"]]["lanes"], recs[c["mmax"]]["threads"])
        out, st = vg.vecchia_batch_loglik_grad_info(*_inputs(bw), bw.offsets, bw.m, cp, bw.covfun,
                                                    handle=h)
        torch.cuda.synchronize()
        assert np.all(st.cpu().numpy()[:, 0] == 0)
        for b in range(bw.nbatch):
            w = bw.dataset(b)
            o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, w.theta_true, w.covfun)
            g = vg.unpack(out[b], 4, 1)
            assert abs(g["loglik"] - o["loglik"]) <= 1e-10 * max(abs(o["loglik"]), w.n)
    finally:
        h.close()

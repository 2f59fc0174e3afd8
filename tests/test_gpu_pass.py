"""GPU parity: the CUDA pass against the FP64 oracle, through the C ABI.

Tolerances (FP64 path): loglik relative 1e-10; gradient ||a-b|| / max(||b||, sqrt(tr info))
<= 1e-10 (the gradient is near zero at an optimum, so it is scaled by the information);
information relative Frobenius 1e-10; betahat ||a-b|| / (||b|| + 1) <= 1e-10."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402

EXP, MAT, ST = vg.EXP_ISO, vg.MATERN_ISO, vg.EXP_SPACETIME
TOL = 1e-10


def compare(g, o, tol=TOL, tol_j=None):
    ll_err = abs(g["loglik"] - o["loglik"]) / abs(o["loglik"])
    scale = max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))
    g_err = np.linalg.norm(g["grad"] - o["grad"]) / scale
    i_err = np.linalg.norm(g["info"] - o["info"]) / np.linalg.norm(o["info"])
    b_err = np.linalg.norm(g["betahat"] - o["betahat"]) / (np.linalg.norm(o["betahat"]) + 1)
    # each component on its own scale too, so that a small one cannot hide under the norm
    # a component whose information is negligible (not identified at this theta) is
    # compared on 1e-4 of the norm scale instead of its own
    gj_scale = np.maximum(np.sqrt(np.abs(np.diag(o["info"]))), 1e-4 * scale)
    gj_err = float(np.max(np.abs(g["grad"] - o["grad"]) / gj_scale))
    errs = dict(loglik=ll_err, grad=g_err, info=i_err, beta=b_err)
    assert max(errs.values()) <= tol, errs
    assert gj_err <= (tol if tol_j is None else tol_j), dict(errs, grad_j=gj_err)
    errs["grad_j"] = gj_err
    return errs


def gpu_pass(w, theta, lanes=0, covfun=None, prec="fp64"):
    dev = torch.device("cuda:0")
    h = vg.Handle(0)
    h.set_lanes(lanes)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    out, st = vg.vecchia_loglik_grad_info(t(w.locs, torch.float64), t(w.y, torch.float64),
                                          t(w.X, torch.float64), t(w.NN, torch.int32),
                                          t(theta, torch.float64),
                                          w.covfun if covfun is None else covfun, prec=prec,
                                          handle=h)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    res = vg.unpack(out, len(theta), w.p)
    res["status"] = int(st[0])
    res["bad_index"] = int(st[1])
    h.close()
    return res


def field(covfun, n, m, p, theta, seed=0, sim="sequential"):
    return workloads.make_field(n, covfun, theta, m, p=p, seed=seed, sim=sim,
                                beta=np.linspace(1.0, -0.5, p), m_sim=min(m + 10, 60))


# ------------------------------------------------------------------ covariance functions
def test_matern_device_covariance_matches_oracle():
    rng = np.random.default_rng(0)
    # below x^2 = 2^-30 the device uses the small-argument expansion (down to 1e-150 here)
    x = np.concatenate([np.geomspace(1e-150, 1e-7, 60, endpoint=False),
                        np.geomspace(1e-7, 95.0, 400), rng.uniform(0, 3, 300)])
    la = np.zeros((len(x), 2))
    lb = np.column_stack([x * 0.7, np.zeros(len(x))])
    same = np.zeros(len(x), np.int32)
    same[:5] = 1
    lb[:5] = 0.0
    dev = torch.device("cuda:0")
    for nu in [0.05, 0.3, 0.5, 0.989, 0.999, 0.9999999, 1.0, 1.0000001, 1.001, 1.0101, 1.5,
               1.9899, 1.999999, 2.0, 2.0000001, 2.5, 4.0, 10.0, 20.0]:
        th = np.array([1.3, 0.7, nu, 0.02])
        C, dC = vg.vecchia_covariance_pairs(
            MAT, torch.tensor(th, device=dev), torch.tensor(la, device=dev),
            torch.tensor(lb, device=dev), torch.tensor(same, device=dev))
        Co, dCo = oracle.cov_pairs(MAT, th, la, lb, same)
        C, dC = C.cpu().numpy(), dC.cpu().numpy()
        assert np.all(np.abs(C - Co) <= 2e-15 * th[0] + 1e-13 * np.abs(Co)), nu
        # derivative scales: dC/dsigma2 ~ 1, dC/drho ~ sigma2/rho, dC/dnu ~ sigma2, dC/dtau2 ~ sigma2.
        # dM/dnu = M (log x - log 2 - psi(nu)) + ... cancels to ~x^(2 nu) log x at small x, so
        # both sides carry ~1e-16 |log x| absolute error there.
        scale = [1.0, th[0] / th[1], 1e2 * th[0], th[0]]
        for j in range(4):
            err = np.abs(dC[:, j] - dCo[:, j])
            assert np.all(err <= 1e-14 * scale[j] + 1e-11 * np.abs(dCo[:, j])), (nu, j, err.max())


def test_covariance_pairs_outside_the_domain_give_nan():
    # parameters are read on the device; a smoothness or range outside the domain must give
    # NaN outputs (finite invalid values only: they end quickly on every code path)
    dev = torch.device("cuda:0")
    la = torch.zeros((4, 2), dtype=torch.float64, device=dev)
    lb = torch.tensor([[0.1, 0.0], [0.3, 0.2], [0.0, 0.0], [1.0, 1.0]], dtype=torch.float64, device=dev)
    same = torch.tensor([0, 0, 1, 0], dtype=torch.int32, device=dev)
    for covfun, th in ((MAT, [1.0, 0.1, -1.0, 0.1]), (MAT, [1.0, 0.1, 25.0, 0.1]),
                       (MAT, [1.0, -0.1, 1.5, 0.1]), (EXP, [1.0, 0.0, 0.1])):
        C, dC = vg.vecchia_covariance_pairs(covfun, torch.tensor(th, dtype=torch.float64, device=dev),
                                            la, lb, same)
        assert torch.isnan(C).all() and torch.isnan(dC).all(), (covfun, th)


# ------------------------------------------------------------------ pass parity
CASES = [
    (EXP, [1.0, 0.1, 0.01], 1, 10),
    (EXP, [0.8, 0.2, 0.1], 2, 30),
    (MAT, [2.0, 0.05, 1.5, 0.05], 3, 30),
    (MAT, [1.2, 0.1, 0.7, 0.02], 1, 20),
    (MAT, [1.0, 0.08, 3.3, 0.1], 2, 12),
    (ST, [1.0, 0.3, 0.4, 0.1], 2, 30),
]


@pytest.mark.parametrize("covfun,theta,p,m", CASES)
def test_pass_matches_oracle(covfun, theta, p, m):
    # several blocks of work and a ragged tail: n not a multiple of any group count
    w = field(covfun, 2377, m, p, theta, seed=3)
    th = np.array(theta)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, covfun)
    g = gpu_pass(w, th)
    assert g["status"] == 0
    compare(g, o)
    # away from the truth as well (start of a fit)
    th2 = th * np.array([1.5, 2.0] + [0.7] * (len(th) - 2))
    compare(gpu_pass(w, th2), oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th2, covfun))


@pytest.mark.parametrize("nu", [0.3, 1.0, 1.0004, 1.5, 2.0, 3.5])
def test_pass_at_extreme_range_matches_oracle(nu):
    # a trial point of a fit that runs off towards rho -> infinity: every scaled squared
    # distance is far below the coefficient table, so each pair takes the small-argument
    # expansion, in the FP64 pass and in the mixed one
    w = field(MAT, 700, 12, 1, [1.0, 0.1, 1.5, 0.05], seed=5)
    th = np.array([0.9, 3.0e4, nu, 0.08])
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, MAT)
    # the smoothness component has almost no information here (the field is nearly
    # constant over the block), and the two sides' expansions of dM/dnu at these tiny
    # arguments agree to ~2e-10 of its scale: the norm check keeps 1e-10, the per-component
    # one 1e-8
    compare(gpu_pass(w, th), o, tol_j=1e-8)
    gm = gpu_pass(w, th, prec="mixed")
    assert gm["status"] == 0
    assert abs(gm["loglik"] - o["loglik"]) <= 1e-4 * max(abs(o["loglik"]), w.n)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("covfun,theta,m,p", [
    (MAT, [1.5, 0.07, 1.2, 0.05], 15, 2),
    (MAT, [1.5, 0.07, 1.2, 0.05], 5, 1),   # small enough for one lane per observation
    (EXP, [1.1, 0.2, 0.05], 8, 1),
])
def test_every_lane_mapping(lanes, covfun, theta, m, p):
    th = np.array(theta)
    w = field(covfun, 900, m, p, th, seed=5)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, covfun)
    try:
        g = gpu_pass(w, th, lanes=lanes)
    except vg.VecchiaError as e:
        assert e.code == 7  # that mapping does not fit shared memory
        assert not (lanes >= 8 and m <= 8)
        return
    compare(g, o)


def test_small_exponential_workload_host_entry_point():
    w = workloads.cfg_small_exp()
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, w.theta_true, w.covfun)
    g = vg.vecchia_loglik_grad_info_host(w.locs, w.y, w.X, w.NN, w.theta_true, w.covfun)
    compare(g, o)


def test_edge_cases_single_point_m0_and_short_rows():
    th = np.array([1.1, 0.2, 0.9, 0.05])
    w = field(MAT, 50, 8, 2, th, seed=8, sim="dense")
    # n = 1 (p = 1; with p = 2 the profile step has a singular X' S^-1 X on both sides)
    w1 = workloads.Workload("one", MAT, w.locs[:1], w.y[:1], np.ascontiguousarray(w.X[:1, :1]),
                            w.NN[:1], th, th, 8)
    compare(gpu_pass(w1, th), oracle.loglik_grad_info(w1.locs, w1.y, w1.X, w1.NN, th, MAT))
    w1b = workloads.Workload("one_p2", MAT, w.locs[:1], w.y[:1], w.X[:1], w.NN[:1], th, th, 8)
    g = gpu_pass(w1b, th)
    assert g["status"] != 0 and np.isnan(g["loglik"])
    with pytest.raises(oracle.OracleError):
        oracle.loglik_grad_info(w1b.locs, w1b.y, w1b.X, w1b.NN, th, MAT)
    # m = 0
    NN0 = np.ascontiguousarray(w.NN[:, :1])
    w0 = workloads.Workload("m0", MAT, w.locs, w.y, w.X, NN0, th, th, 0)
    compare(gpu_pass(w0, th), oracle.loglik_grad_info(w.locs, w.y, w.X, NN0, th, MAT))
    # rows with fewer neighbours than min(i, m): drop the farthest ones at random
    NNs = w.NN.copy()
    rng = np.random.default_rng(1)
    for i in range(len(NNs)):
        k = int((NNs[i, 1:] >= 0).sum())
        keep = rng.integers(0, k + 1) if k else 0
        NNs[i, 1 + keep:] = -1
    ws = workloads.Workload("short", MAT, w.locs, w.y, w.X, NNs, th, th, 8)
    compare(gpu_pass(ws, th), oracle.loglik_grad_info(w.locs, w.y, w.X, NNs, th, MAT))


def test_largest_m_and_p():
    th = np.array([1.0, 0.15, 0.05])
    w = field(EXP, 700, 80, 1, th, seed=2, sim="dense")
    x1, x2 = w.locs[:, 0], w.locs[:, 1]
    # eight linearly independent regressors: a cubic surface without the x1^2 x2, x1 x2^2 terms
    X = np.column_stack([np.ones(w.n), x1, x2, x1 * x1, x1 * x2, x2 * x2, x1 ** 3, x2 ** 3])
    w8 = workloads.Workload("p8", EXP, w.locs, w.y + X @ np.linspace(0.5, -0.5, 8), X, w.NN,
                            th, th, 80)
    o = oracle.loglik_grad_info(w8.locs, w8.y, w8.X, w8.NN, th, EXP)
    compare(gpu_pass(w8, th), o)


def test_errors_are_reported_not_faulted():
    th = np.array([1.0, 0.1, 1.5, 0.05])
    w = field(MAT, 300, 10, 1, th, seed=4, sim="dense")
    # covariance parameter out of range
    g = gpu_pass(w, np.array([1.0, 0.1, 25.0, 0.05]))
    assert g["status"] == 1 and np.isnan(g["loglik"])
    g = gpu_pass(w, np.array([-1.0, 0.1, 1.5, 0.05]))
    assert g["status"] == 1
    # a neighbour that is not earlier
    NN = w.NN.copy()
    NN[200, 1] = 250
    wb = workloads.Workload("bad", MAT, w.locs, w.y, w.X, NN, th, th, 10)
    g = gpu_pass(wb, th)
    assert g["status"] == 1 and g["bad_index"] == 200
    # a singular block: a point on top of its nearest neighbour, smooth field, no nugget
    locs = w.locs.copy()
    locs[150] = locs[w.NN[150, 1]]
    thx = np.array([1.0, 1.0, 20.0, 1e-300])
    wx = workloads.Workload("npd", MAT, locs, w.y, w.X, w.NN, thx, thx, 10)
    g = gpu_pass(wx, thx)
    assert g["status"] == 2 and 0 <= g["bad_index"] <= 150
    with pytest.raises(vg.VecchiaError) as e:
        vg.vecchia_loglik_grad_info_host(locs, w.y, w.X, w.NN, thx, MAT)
    assert e.value.code == 2


def test_repeat_runs_are_bitwise_identical():
    th = np.array([2.0, 0.05, 1.5, 0.05])
    w = field(MAT, 3000, 30, 3, th, seed=6)
    a = gpu_pass(w, th)
    b = gpu_pass(w, th)
    assert a["loglik"] == b["loglik"] and np.array_equal(a["grad"], b["grad"])
    assert np.array_equal(a["info"], b["info"])


@pytest.mark.slow
def test_full_size_matern_100k_matches_oracle():
    """The n = 1e5, m = 30 Matern workload in the same launch configuration the benchmark
    times, at the true and at the starting parameters."""
    w = workloads.cfg_matern_100k()
    for th in (w.theta_true, w.theta_start):
        o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, w.covfun)
        compare(gpu_pass(w, th), o)


@pytest.mark.slow
@pytest.mark.parametrize("placement", ["global", "shared"])
def test_full_size_matern_100k_each_table_placement(placement):
    """The full-size pass with the mappings the autotuner picks on GB300 for FP64 (16 lanes,
    96 threads) and for mixed precision (16 lanes, 192 threads), then FP64 with 8 lanes and
    64 threads, with the Matern table in global and in shared memory; the FP64 passes
    against the oracle, the mixed one within its bounds."""
    w = workloads.cfg_matern_100k()
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, w.theta_true, w.covfun)
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    args = (t(w.locs, torch.float64), t(w.y, torch.float64), t(w.X, torch.float64),
            t(w.NN, torch.int32), t(w.theta_true, torch.float64), w.covfun)
    for prec, lanes, threads in (("fp64", 16, 96), ("mixed", 16, 192), ("fp64", 8, 64)):
        h = vg.Handle(0)
        h.set_lanes(lanes)
        h.set_block_threads(threads)
        h.set_matern_table(placement)
        out, st = vg.vecchia_loglik_grad_info(*args, prec=prec, handle=h)
        torch.cuda.synchronize()
        h.close()
        assert int(st[0]) == 0
        g = vg.unpack(out, 4, w.p)
        if prec == "fp64":
            compare(g, o)
        else:
            assert abs(g["loglik"] - o["loglik"]) <= 1e-6 * abs(o["loglik"])


@pytest.mark.slow
def test_full_size_swath_matches_oracle():
    """The 1.2 M-point space-time swath workload at full size (m = 30): the FP64 pass at the
    true and the starting parameters against the oracle (1e-10), the mixed pass within the
    stated bounds (tau2 = 0.1), and the FP64 and mixed fits against the oracle's fit."""
    w = workloads.cfg_swath_1m2()
    for th in (w.theta_true, w.theta_start):
        o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, th, w.covfun)
        compare(gpu_pass(w, th), o)
        gm = gpu_pass(w, th, prec="mixed")
        assert abs(gm["loglik"] - o["loglik"]) <= 1e-6 * abs(o["loglik"])
        scale = max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))
        assert np.linalg.norm(gm["grad"] - o["grad"]) <= 2e-4 * scale
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    args = (t(w.locs, torch.float64), t(w.y, torch.float64), t(w.X, torch.float64),
            t(w.NN, torch.int32), w.covfun, w.theta_start)
    of = oracle.fisher_fit(w.locs, w.y, w.X, w.NN, w.covfun, w.theta_start)
    g64 = vg.vecchia_fit(*args)
    gmx = vg.vecchia_fit(*args, prec="mixed")
    assert g64["status"] == of["status"] == 0 and gmx["status"] == 0
    assert g64["iters"] == of["iters"]
    assert abs(g64["loglik"] - of["loglik"]) <= 1e-8 * abs(of["loglik"])
    assert abs(gmx["loglik"] - of["loglik"]) <= 1e-8 * abs(of["loglik"])

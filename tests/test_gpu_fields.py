"""Fields at shared locations: the simulation equals the oracle's sequential draw (Sec. 2.1,
Eq. 3) for the same variates, and the pass and the fit equal the batched calls on the same
data with the geometry replicated per field (same kernels, same tiles: bitwise)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import simulate as osim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402

EXP, MAT = vg.EXP_ISO, vg.MATERN_ISO


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=torch.device("cuda:0"))


def _geometry(n, m, seed):
    L = np.random.default_rng(seed).uniform(size=(n, 2))
    L = L[workloads.maxmin_order(L)]
    return L, workloads.ordered_nn(L, m)


@pytest.mark.parametrize("covfun,thetas", [
    (MAT, [[1.0, 0.1, 1.5, 0.05], [0.6, 0.05, 0.7, 0.01], [1.8, 0.2, 2.2, 0.2]]),
    (EXP, [[1.0, 0.1, 0.01], [2.0, 0.3, 0.1]]),
])
def test_simulate_matches_oracle(covfun, thetas):
    n, m = 700, 12
    locs, NN = _geometry(n, m, 1)
    th = np.array(thetas)
    z = np.random.default_rng(2).standard_normal((len(th), n))
    y, st = vg.vecchia_fields_simulate(_dev(locs, torch.float64), _dev(NN, torch.int32),
                                       _dev(th, torch.float64), covfun, _dev(z, torch.float64))
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy()[:, 0] == 0)
    y = y.cpu().numpy()
    for b in range(len(th)):
        yo = osim.simulate(locs, NN, th[b], covfun, z[b])
        assert np.max(np.abs(y[b] - yo)) <= 1e-10 * np.max(np.abs(yo))


def test_simulate_reports_bad_parameters_per_field():
    n, m = 300, 8
    locs, NN = _geometry(n, m, 3)
    th = np.array([[1.0, 0.1, 1.5, 0.05], [1.0, -0.1, 1.5, 0.05], [1.0, 0.1, 1.5, 0.05]])
    z = np.random.default_rng(4).standard_normal((3, n))
    z[2] = z[0]
    y, st = vg.vecchia_fields_simulate(_dev(locs, torch.float64), _dev(NN, torch.int32),
                                       _dev(th, torch.float64), MAT, _dev(z, torch.float64))
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert list(st[:, 0]) == [0, 1, 0]
    assert torch.equal(y[0], y[2])   # same parameters, same variates


def _replicated(locs, NN, Y):
    nf, n = Y.shape
    m = NN.shape[1] - 1
    bl = np.tile(locs, (nf, 1))
    bNN = np.tile(NN.ravel(), nf)
    off = np.arange(nf + 1, dtype=np.int64) * n
    return bl, bNN, off, np.full(nf, m, dtype=np.int32)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fields_pass_and_fit_equal_replicated_batch(prec):
    n, m, nf = 900, 10, 5
    locs, NN = _geometry(n, m, 5)
    rng = np.random.default_rng(6)
    th = np.column_stack([rng.uniform(0.5, 2, nf), rng.uniform(0.03, 0.2, nf),
                          rng.uniform(0.5, 2.5, nf), rng.uniform(0.01, 0.2, nf)])
    z = rng.standard_normal((nf, n))
    dl, dNN = _dev(locs, torch.float64), _dev(NN, torch.int32)
    Y, st = vg.vecchia_fields_simulate(dl, dNN, _dev(th, torch.float64), MAT, _dev(z, torch.float64))
    X = torch.ones(n, 1, dtype=torch.float64, device="cuda:0")
    h = vg.Handle(0)
    h.set_lanes(8)
    h.set_block_threads(128)
    try:
        cp = _dev(th, torch.float64)
        fo, fst = vg.vecchia_fields_loglik_grad_info(dl, X, dNN, Y, cp, MAT, prec=prec, handle=h)
        bl, bNN, off, mm = _replicated(locs, NN, Y.cpu().numpy())
        bo, bst = vg.vecchia_batch_loglik_grad_info(
            _dev(bl, torch.float64), Y.reshape(-1), torch.ones(nf * n, 1, dtype=torch.float64,
                                                               device="cuda:0"),
            _dev(bNN, torch.int32), off, mm, cp, MAT, prec=prec, handle=h)
        torch.cuda.synchronize()
        assert torch.equal(fst, bst) and torch.equal(fo, bo)
        start = torch.tensor([[float(np.var(Y[b].cpu().numpy())), 0.1, 1.0, 0.1] for b in range(nf)],
                             dtype=torch.float64, device="cuda:0")
        ff = vg.vecchia_fields_fit(dl, X, dNN, Y, MAT, start, prec=prec, handle=h)
        bf = vg.vecchia_batch_fit(_dev(bl, torch.float64), Y.reshape(-1),
                                  torch.ones(nf * n, 1, dtype=torch.float64, device="cuda:0"),
                                  _dev(bNN, torch.int32), off, mm, MAT, start, prec=prec, handle=h)
        assert torch.equal(ff["theta"], bf["theta"]) and torch.equal(ff["out"], bf["out"])
        assert np.array_equal(ff["iters"], bf["iters"])
    finally:
        h.close()


def test_fields_pass_matches_oracle():
    n, m, nf = 800, 15, 3
    locs, NN = _geometry(n, m, 7)
    th = np.array([[1.2, 0.08, 1.1, 0.03], [0.7, 0.15, 0.6, 0.1], [1.5, 0.05, 2.0, 0.02]])
    z = np.random.default_rng(8).standard_normal((nf, n))
    Yo = np.array([osim.simulate(locs, NN, th[b], MAT, z[b]) for b in range(nf)])
    Xo = np.column_stack([np.ones(n), locs[:, 0]])
    out, st = vg.vecchia_fields_loglik_grad_info(_dev(locs, torch.float64), _dev(Xo, torch.float64),
                                                 _dev(NN, torch.int32), _dev(Yo, torch.float64),
                                                 _dev(th, torch.float64), MAT)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy()[:, 0] == 0)
    for b in range(nf):
        g = vg.unpack(out[b], 4, 2)
        o = oracle.loglik_grad_info(locs, Yo[b], Xo, NN, th[b], MAT)
        assert abs(g["loglik"] - o["loglik"]) <= 1e-10 * abs(o["loglik"])
        scale = max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))
        assert np.linalg.norm(g["grad"] - o["grad"]) <= 1e-10 * scale
        assert np.all(np.abs(g["grad"] - o["grad"]) <= 1e-10 * np.maximum(
            np.sqrt(np.abs(np.diag(o["info"]))), 1e-4 * max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))))

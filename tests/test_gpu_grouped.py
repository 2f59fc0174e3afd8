"""Grouped conditioning on the device against the oracle (oracle/grouped.py: each group's
terms as differences of dense Gaussian blocks), FP64 to 1e-10 as for the plain pass, at
every lane mapping; singleton groups against the plain device pass; the mixed pass within
its stated bounds; a full-size field against the C oracle's plain pass on the equivalent
expanded NNarray, in one launch and in launch classes by block size; errors."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import grouped as og

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402

EXP, MAT, ST = vg.EXP_ISO, vg.MATERN_ISO, vg.EXP_SPACETIME
MIXED_BOUNDS = {"loglik": 1e-6, "grad": 2e-4, "info": 2e-5, "beta": 5e-6}


def _dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=torch.device("cuda:0"))


def _errors(g, o):
    scale = max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))
    return {"loglik": abs(g["loglik"] - o["loglik"]) / abs(o["loglik"]),
            "grad": np.linalg.norm(g["grad"] - o["grad"]) / scale,
            "grad_j": float(np.max(np.abs(g["grad"] - o["grad"]) / np.maximum(
                np.sqrt(np.abs(np.diag(o["info"]))), 1e-4 * max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"])))))),
            "info": np.linalg.norm(g["info"] - o["info"]) / np.linalg.norm(o["info"]),
            "beta": np.linalg.norm(g["betahat"] - o["betahat"]) / (np.linalg.norm(o["betahat"]) + 1)}


def _grouped(w, goff, th, lanes=0, prec="fp64", blocks=None, nclass=0, chunk=0):
    off, idx, nm, kmax = blocks if blocks is not None else vg.vecchia_group_blocks(w.NN, goff)
    classes = None
    if nclass:
        gorder, coff, ckmax = vg.vecchia_group_classes(off, nclass)
        classes = (_dev(gorder, torch.int32), coff, ckmax)
    h = vg.Handle(0)
    h.set_lanes(lanes)
    h.set_group_chunk(chunk)
    try:
        out, st = vg.vecchia_grouped_loglik_grad_info(
            _dev(w.locs), _dev(w.y), _dev(w.X), _dev(off, torch.int64), _dev(idx, torch.int32),
            _dev(nm, torch.int32), kmax, _dev(th), w.covfun, prec=prec, handle=h, classes=classes)
        torch.cuda.synchronize()
        r = vg.unpack(out, len(th), w.p)
        r["status"], r["bad"] = int(st[0]), int(st[1])
    finally:
        h.close()
    return r


CASES = [(EXP, [1.2, 0.15, 0.05], 1, 1200, 20, 6), (MAT, [1.1, 0.1, 0.8, 0.03], 2, 900, 30, 8),
         (MAT, [2.0, 0.05, 1.5, 0.05], 3, 1000, 15, 4), (ST, [1.0, 0.3, 0.5, 0.1], 2, 800, 25, 8)]


@pytest.mark.parametrize("covfun,theta,p,n,m,g", CASES)
def test_fp64_matches_oracle(covfun, theta, p, n, m, g):
    w, goff = workloads.grouped_field(n, covfun, theta, m, g, p=p, seed=11, m_sim=min(m + 5, 40),
                                      beta=np.linspace(1.0, -0.5, p))
    th = np.array(theta)
    off, idx, nm = og.group_blocks(w.NN, goff)
    o = og.loglik_grad_info(w.locs, w.y, w.X, off, idx, nm, th, covfun)
    for L in ([0, 4, 8, 16, 32] if covfun == MAT and p == 2 else [0]):
        r = _grouped(w, goff, th, lanes=L)
        assert r["status"] == 0
        e = _errors(r, o)
        assert max(e.values()) <= 1e-10, (L, e)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_members_formed_together_in_any_number(prec):
    # the members' terms formed 1, 2, 3, 5 or 8 at a time (groups of up to 8 members: full
    # chunks, a shorter last chunk, one chunk for the whole group): FP64 against the oracle,
    # mixed within its bounds
    covfun, theta, p, n, m, g = CASES[1]
    w, goff = workloads.grouped_field(n, covfun, theta, m, g, p=p, seed=11, m_sim=min(m + 5, 40),
                                      beta=np.linspace(1.0, -0.5, p))
    th = np.array(theta)
    off, idx, nm = og.group_blocks(w.NN, goff)
    o = og.loglik_grad_info(w.locs, w.y, w.X, off, idx, nm, th, covfun)
    for chunk in (1, 2, 3, 5, 8):
        r = _grouped(w, goff, th, lanes=32, prec=prec, chunk=chunk)
        assert r["status"] == 0
        e = _errors(r, o)
        if prec == "fp64":
            assert max(e.values()) <= 1e-10, (chunk, e)
        else:
            assert all(e[k] <= MIXED_BOUNDS[k] for k in MIXED_BOUNDS), (chunk, e)


@pytest.mark.parametrize("nclass", [2, 3])
def test_launch_classes_give_the_same_result(nclass):
    th = np.array([1.1, 0.1, 0.8, 0.03])
    w, goff = workloads.grouped_field(1500, MAT, th, 30, 8, p=2, seed=16, m_sim=30,
                                      beta=[1.0, -0.5])
    off, idx, nm, kmax = vg.vecchia_group_blocks(w.NN, goff)
    one = _grouped(w, goff, th, blocks=(off, idx, nm, kmax))
    gorder, coff, ckmax = vg.vecchia_group_classes(off, nclass)
    h = vg.Handle(0)
    try:
        out, st = vg.vecchia_grouped_loglik_grad_info(
            _dev(w.locs), _dev(w.y), _dev(w.X), _dev(off, torch.int64), _dev(idx, torch.int32),
            _dev(nm, torch.int32), kmax, _dev(th), MAT, handle=h,
            classes=(_dev(gorder, torch.int32), coff, ckmax))
        torch.cuda.synchronize()
    finally:
        h.close()
    assert int(st[0]) == 0
    g = vg.unpack(out, 4, 2)
    e = _errors(g, one)
    assert max(e.values()) <= 1e-12, e
    o = og.loglik_grad_info(w.locs, w.y, w.X, off, idx, nm, th, MAT)
    assert max(_errors(g, o).values()) <= 1e-10


def test_singleton_groups_equal_the_plain_pass():
    th = np.array([1.3, 0.08, 1.2, 0.05])
    w, _ = workloads.grouped_field(3000, MAT, th, 30, 8, p=2, seed=12, m_sim=30)
    r = _grouped(w, np.arange(w.n + 1), th)
    out, st = vg.vecchia_loglik_grad_info(_dev(w.locs), _dev(w.y), _dev(w.X), _dev(w.NN, torch.int32),
                                          _dev(th), MAT)
    torch.cuda.synchronize()
    g = vg.unpack(out, 4, 2)
    e = _errors(r, g)
    assert max(e.values()) <= 1e-12, e


def test_mixed_within_stated_bounds():
    th = np.array([1.1, 0.1, 0.8, 0.05])
    w, goff = workloads.grouped_field(1500, MAT, th, 20, 6, p=1, seed=13, m_sim=25)
    off, idx, nm = og.group_blocks(w.NN, goff)
    o = og.loglik_grad_info(w.locs, w.y, w.X, off, idx, nm, th, MAT)
    r = _grouped(w, goff, th, prec="mixed")
    assert r["status"] == 0
    e = _errors(r, o)
    assert all(e[k] <= MIXED_BOUNDS[k] for k in MIXED_BOUNDS), e


def _expanded_nn(off, idx, nm):
    rows = []
    for b in range(len(off) - 1):
        blk = list(idx[off[b]:off[b + 1]])
        nu = len(blk) - nm[b]
        for r in range(nu, len(blk)):
            rows.append([blk[r]] + blk[:r][::-1])
    W = max(len(r) for r in rows)
    return np.array([r + [-1] * (W - len(r)) for r in rows], dtype=np.int32)


@pytest.mark.slow
def test_full_size_against_the_expanded_plain_oracle():
    # n = 1e5 Matern field in groups of about 8: the grouped density is the plain Vecchia
    # density on the expanded NNarray (member i conditions on U and the earlier members)
    th = np.array([2.0, 0.05, 1.5, 0.05])
    w, goff = workloads.grouped_field(100000, MAT, th, 30, 8, p=3, seed=14, m_sim=30,
                                      beta=[1.0, 0.5, -0.5])
    blocks = vg.vecchia_group_blocks(w.NN, goff)
    NNx = _expanded_nn(*blocks[:3])
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, NNx, th, MAT)
    r = _grouped(w, goff, th, blocks=blocks)
    assert r["status"] == 0
    e = _errors(r, o)
    assert max(e.values()) <= 1e-10, e
    # the same groups in three launches by block size (slots sized per class)
    r = _grouped(w, goff, th, blocks=blocks, nclass=3)
    assert r["status"] == 0
    e = _errors(r, o)
    assert max(e.values()) <= 1e-10, e


def test_errors():
    th = np.array([1.0, 0.1, 1.0, 0.05])
    w, goff = workloads.grouped_field(400, MAT, th, 10, 4, seed=15, m_sim=10)
    off, idx, nm, kmax = vg.vecchia_group_blocks(w.NN, goff)
    bad = idx.copy()
    b = 7
    s = off[b] + (off[b + 1] - off[b]) - nm[b]     # the first member of block 7
    bad[s - 1] = bad[s] + 1 if s > off[b] else bad[s]
    r = _grouped(w, goff, th, blocks=(off, bad, nm, kmax))
    assert r["status"] == 1 and r["bad"] >= 0 and np.isnan(r["loglik"])
    with pytest.raises(vg.VecchiaError):
        _grouped(w, goff, th, blocks=(off, idx, nm, 90))     # kmax above the largest block size
    w2 = workloads.make_field(200, vg.EXP_ANISO, [1.0, 0.3, 0.4, 0.1], 5, seed=1)
    with pytest.raises(vg.VecchiaError):
        _grouped(w2, np.arange(w2.n + 1), np.array([1.0, 0.3, 0.4, 0.1]))

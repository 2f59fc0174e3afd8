"""Pins for the grouped-conditioning oracle (oracle/grouped.py), each against something
other than itself:
  * singleton groups are plain Vecchia: equal to the C oracle's Algorithm 1 pass;
  * one group holding every observation (no conditioning set) is the exact Gaussian
    likelihood, gradient and Fisher information (dense, as in test_oracle_pass);
  * in general the grouped density is the Vecchia density whose member i conditions on
    U_b and the earlier members of its group: its loglik is that of the dense density
    implied by those conditionals, and its gradient matches central differences of it;
  * the blocks: U_b precedes the group, holds exactly the members' other neighbours."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import grouped as og
from test_oracle_pass import dense_gp, implied_loglik

EXP, MAT, ST = oracle.EXP_ISO, oracle.MATERN_ISO, oracle.EXP_SPACETIME


def _field(covfun, theta, n, m, g, p, seed):
    return workloads.grouped_field(n, covfun, theta, m, g, p=p, seed=seed, m_sim=min(m + 5, 40),
                                   beta=np.linspace(0.5, -0.5, p))


def _expanded_nn(w, goff):
    """NNarray of the equivalent ungrouped density: member i conditions on U_b and the
    earlier members of its group."""
    off, idx, nm = og.group_blocks(w.NN, goff)
    rows = []
    for b in range(len(goff) - 1):
        blk = list(idx[off[b]:off[b + 1]])
        nu = len(blk) - nm[b]
        for r in range(nu, len(blk)):
            rows.append([blk[r]] + sorted(blk[:r], reverse=True))
    W = max(len(r) for r in rows)
    return np.array([r + [-1] * (W - len(r)) for r in rows], dtype=np.int32)


CASES = [(EXP, [1.2, 0.15, 0.05], 1), (MAT, [1.1, 0.1, 0.8, 0.03], 2), (ST, [1.0, 0.3, 0.5, 0.1], 2)]


@pytest.mark.parametrize("covfun,theta,p", CASES)
def test_singleton_groups_are_plain_vecchia(covfun, theta, p):
    w, _ = _field(covfun, theta, 150, 8, 5, p, seed=1)
    off, idx, nm = og.group_blocks(w.NN, np.arange(w.n + 1))
    g = og.loglik_grad_info(w.locs, w.y, w.X, off, idx, nm, theta, covfun)
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, np.array(theta), covfun)
    assert abs(g["loglik"] - o["loglik"]) <= 1e-11 * abs(o["loglik"])
    assert np.allclose(g["grad"], o["grad"], rtol=1e-9, atol=1e-9 * np.abs(o["grad"]).max())
    assert np.allclose(g["info"], o["info"], rtol=1e-9, atol=1e-9 * np.abs(o["info"]).max())


@pytest.mark.parametrize("covfun,theta,p", CASES)
def test_one_group_is_the_exact_likelihood(covfun, theta, p):
    w, _ = _field(covfun, theta, 70, 8, 5, p, seed=2)
    off, idx, nm = og.group_blocks(w.NN, np.array([0, w.n]))
    assert list(idx) == list(range(w.n))
    g = og.loglik_grad_info(w.locs, w.y, w.X, off, idx, nm, theta, covfun)
    ll, grad, info, beta = dense_gp(covfun, np.array(theta), w.locs, w.y, w.X)
    assert abs(g["loglik"] - ll) <= 1e-11 * abs(ll)
    scale = max(np.linalg.norm(grad), np.sqrt(np.trace(info)))
    assert np.linalg.norm(g["grad"] - grad) <= 1e-10 * scale
    assert np.linalg.norm(g["info"] - info) <= 1e-10 * np.linalg.norm(info)


@pytest.mark.parametrize("covfun,theta,p", CASES)
def test_grouped_density_is_the_implied_density(covfun, theta, p):
    w, goff = _field(covfun, theta, 160, 6, 6, p, seed=3)
    off, idx, nm = og.group_blocks(w.NN, goff)
    th = np.array(theta)
    g = og.loglik_grad_info(w.locs, w.y, w.X, off, idx, nm, th, covfun)
    NNx = _expanded_nn(w, goff)
    ll, beta = implied_loglik(covfun, th, w.locs, w.y, w.X, NNx)
    assert abs(g["loglik"] - ll) <= 1e-11 * abs(ll)
    assert np.linalg.norm(g["betahat"] - beta) <= 1e-10 * (np.linalg.norm(beta) + 1)
    fd = np.empty(len(th))
    for j in range(len(th)):
        h = 1e-5 * th[j]
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd[j] = (implied_loglik(covfun, tp, w.locs, w.y, w.X, NNx)[0]
                 - implied_loglik(covfun, tm, w.locs, w.y, w.X, NNx)[0]) / (2 * h)
    scale = max(np.linalg.norm(fd), np.sqrt(np.trace(g["info"])))
    assert np.linalg.norm(g["grad"] - fd) <= 1e-6 * scale
    # and the same density through the C oracle's plain pass on the expanded NNarray
    o = oracle.loglik_grad_info(w.locs, w.y, w.X, NNx, th, covfun)
    assert abs(g["loglik"] - o["loglik"]) <= 1e-11 * abs(o["loglik"])
    assert np.allclose(g["info"], o["info"], rtol=1e-9, atol=1e-9 * np.abs(o["info"]).max())


def test_blocks_and_groups():
    w, goff = _field(MAT, [1.0, 0.1, 1.0, 0.05], 3000, 30, 8, 1, seed=4)
    assert goff[0] == 0 and goff[-1] == w.n and np.all(np.diff(goff) >= 1)
    assert np.all(np.diff(goff) <= 16)
    off, idx, nm = og.group_blocks(w.NN, goff)
    for b in range(len(goff) - 1):
        s, e = goff[b], goff[b + 1]
        blk = idx[off[b]:off[b + 1]]
        U, B = blk[:len(blk) - nm[b]], blk[len(blk) - nm[b]:]
        assert list(B) == list(range(s, e))
        assert np.all(U < s) and np.all(np.diff(U) > 0)
        want = set(int(j) for i in range(s, e) for j in w.NN[i, 1:] if j >= 0) - set(range(s, e))
        assert set(int(j) for j in U) == want
    # compact groups share neighbours: blocks stay far below members x (m + 1)
    K = np.diff(off)
    assert K.max() <= 81 and K.mean() < 0.5 * np.mean(nm) * 31

"""The learned-start network's kernels against the FP64 oracle: forward predictions,
loss and gradient (FP32 vs FP64: 1e-4 relative in norm), the Adam update, column
moments, determinism, ragged sample counts, and a training run that fits a smooth
target function."""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2407_02740_gb300 as vg  # noqa: E402


def _f32(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda:0")


def _setup(B, seed):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(rng).astype(np.float32)
    params[-4:] = rng.standard_normal(4).astype(np.float32) * 0.1
    norm = np.concatenate([rng.standard_normal(32), rng.uniform(0.5, 2, 32),
                           rng.standard_normal(4), rng.uniform(0.5, 2, 4)]).astype(np.float32)
    X = rng.standard_normal((B, 32)).astype(np.float32)
    T = rng.standard_normal((B, 4)).astype(np.float32)
    return params, norm, X, T


@pytest.mark.parametrize("B", [1, 32, 77, 1000])
def test_forward_and_gradient_match_oracle(B):
    params, norm, X, T = _setup(B, B)
    pred = vg.vecchia_mlp_forward(_f32(params), _f32(norm), _f32(X)).cpu().numpy()
    po = mlp.forward(params, norm, X)
    assert np.allclose(pred, po, rtol=1e-4, atol=1e-4 * np.abs(po).max())
    g, loss = vg.vecchia_mlp_grad(_f32(params), _f32(norm), _f32(X), _f32(T))
    lo, go = mlp.loss_grad(params, norm, X, T)
    g = g.cpu().numpy()
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)


def test_gradient_is_deterministic_and_index_selects_rows():
    params, norm, X, T = _setup(500, 7)
    a = vg.vecchia_mlp_grad(_f32(params), _f32(norm), _f32(X), _f32(T))
    b = vg.vecchia_mlp_grad(_f32(params), _f32(norm), _f32(X), _f32(T))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    idx = np.random.default_rng(8).permutation(500)[:123].astype(np.int32)
    gi, li = vg.vecchia_mlp_grad(_f32(params), _f32(norm), _f32(X), _f32(T),
                                 index=torch.as_tensor(idx, device="cuda:0"))
    lo, go = mlp.loss_grad(params, norm, X[idx], T[idx])
    assert abs(float(li.item()) - lo) <= 1e-5 * lo
    assert np.linalg.norm(gi.cpu().numpy() - go) <= 1e-4 * np.linalg.norm(go)


def test_adam_steps_match_oracle():
    params, norm, X, T = _setup(200, 3)
    P = _f32(params)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    po, mo, vo = params.astype(np.float64), np.zeros(len(params)), np.zeros(len(params))
    for step in (1, 2, 3):
        _, go = mlp.loss_grad(po, norm, X, T)
        po, mo, vo = mlp.adam_step(po, mo, vo, go, step, 1e-3)
        vg.vecchia_mlp_adam_step(P, m, v, step, 1e-3, _f32(norm), _f32(X), _f32(T))
    d = P.cpu().numpy() - po
    # each step moves a parameter by at most ~lr; FP32 gradients can flip a tiny update
    assert np.abs(d).max() <= 3e-3 and np.mean(np.abs(d)) <= 2e-5


def test_column_moments():
    X = np.random.default_rng(1).standard_normal((5000, 36)).astype(np.float32) * 3 + 1
    X[:, 5] = 2.0
    mu, sd = vg.vecchia_mlp_column_moments(_f32(X))
    mu, sd = mu.cpu().numpy(), sd.cpu().numpy()
    assert np.allclose(mu, X.astype(np.float64).mean(axis=0), rtol=1e-6, atol=1e-6)
    ref = X.astype(np.float64).std(axis=0)
    ref[5] = 1.0
    assert np.allclose(sd, ref, rtol=1e-6)


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((4096, 32)).astype(np.float32)
    A = rng.standard_normal((32, 4)) / 6
    T = (np.tanh(X @ A) + 0.3 * (X[:, :4] ** 2)).astype(np.float32)
    xm, xs = vg.vecchia_mlp_column_moments(_f32(X))
    tm, ts = vg.vecchia_mlp_column_moments(_f32(T))
    norm = torch.cat([xm, xs, tm, ts])
    P = _f32(mlp.init_params(rng))
    m, v = torch.zeros_like(P), torch.zeros_like(P)
    Xd, Td = _f32(X), _f32(T)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    losses = []
    step = 0
    for epoch in range(40):
        perm = torch.as_tensor(rng.permutation(4096).astype(np.int32), device="cuda:0")
        for b in range(0, 4096, 256):
            step += 1
            vg.vecchia_mlp_adam_step(P, m, v, step, 2e-3, norm, Xd, Td, index=perm[b:b + 256],
                                     loss=loss)
        losses.append(float(loss.item()))
    assert losses[-1] < 0.1 * losses[0]


def test_field_moments_targets_and_theta_from_predictions():
    # the learned start's per-field steps against their definitions in numpy (FP64)
    rng = np.random.default_rng(11)
    nf, n = 37, 1001
    Y = rng.normal(size=(nf, n)) * rng.uniform(0.2, 3.0, (nf, 1)) + rng.normal(size=(nf, 1))
    Yd = torch.as_tensor(Y, device="cuda:0")
    mean, var = vg.vecchia_fields_moments(Yd)
    assert np.allclose(mean.cpu().numpy(), Y.mean(axis=1), rtol=1e-13, atol=1e-14)
    assert np.allclose(var.cpu().numpy(), Y.var(axis=1), rtol=1e-13)
    theta = np.column_stack([rng.uniform(0.1, 5, nf), np.exp(rng.uniform(-12, 3, nf)),
                             rng.uniform(0.06, 19, nf), np.exp(rng.uniform(-16, 3, nf))])
    lo, hi = [1e-2, 1e-4, 0.05, 1e-6], [1e2, 1e1, 20.0, 1e1]
    T = vg.vecchia_mlp_targets(torch.as_tensor(theta, device="cuda:0"), var, lo, hi).cpu().numpy()
    ref = np.log(theta)
    ref[:, 0] -= np.log(Y.var(axis=1))
    ref = np.clip(ref, np.log(lo), np.log(hi)).astype(np.float32)
    assert np.allclose(T, ref, rtol=1e-6, atol=1e-6)
    pred = rng.normal(size=(nf, 4)).astype(np.float32) * 2
    pred[:3, 2] = [-4.0, 4.0, 0.0]            # nu below and above the clamp
    th0 = vg.vecchia_mlp_theta(_f32(pred), var).cpu().numpy()
    want = np.exp(pred.astype(np.float64))
    want[:, 0] *= Y.var(axis=1)
    want[:, 2] = np.clip(want[:, 2], 0.05, 20.0)
    assert np.allclose(th0, want, rtol=1e-13)

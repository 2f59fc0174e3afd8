"""Pins for the learned-start network oracle: the backward pass against central finite
differences of the loss, closed forms of the output layer and of the first Adam step."""
import numpy as np

from oracle import mlp


def _setup(B=13, seed=0):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(rng)
    params[mlp.NPARAMS - 4:] = rng.standard_normal(4) * 0.1
    norm = np.concatenate([rng.standard_normal(32), rng.uniform(0.5, 2, 32),
                           rng.standard_normal(4), rng.uniform(0.5, 2, 4)])
    X = rng.standard_normal((B, 32))
    T = rng.standard_normal((B, 4))
    return rng, params, norm, X, T


def test_gradient_matches_central_differences():
    rng, params, norm, X, T = _setup()
    _, g = mlp.loss_grad(params, norm, X, T)
    idx = np.concatenate([rng.choice(4096, 40, replace=False),            # W1
                          4096 + rng.choice(128, 10, replace=False),      # b1
                          4224 + rng.choice(16384, 60, replace=False),    # W2
                          20608 + rng.choice(128, 10, replace=False),     # b2
                          20736 + rng.choice(512, 20, replace=False),     # W3
                          21248 + np.arange(4)])                          # b3
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        fd = (mlp.loss_grad(params + e, norm, X, T)[0] - mlp.loss_grad(params - e, norm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_output_layer_closed_forms():
    _, params, norm, X, T = _setup()
    P = params.copy()
    P[20736:21248] = 0.0            # W3 = 0: the output is b3 whatever the input
    b3 = P[21248:]
    pred = mlp.forward(P, norm, X)
    assert np.allclose(pred, b3 * norm[68:72] + norm[64:68], rtol=1e-15)
    t = (T - norm[64:68]) / norm[68:72]
    loss, g = mlp.loss_grad(P, norm, X, T)
    assert np.isclose(loss, np.mean((b3 - t) ** 2), rtol=1e-14)
    assert np.allclose(g[21248:], 2.0 * (b3 - t).mean(axis=0) / 4, rtol=1e-13)
    assert np.all(g[:20736] == 0.0)  # no signal reaches the hidden layers


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    p1, m, v = mlp.adam_step(p, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    # bias-corrected moments at step 1 are g and g^2
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)

"""Oracle for the learned-start network -- TEST INFRASTRUCTURE (see ``oracle/__init__``).

32 -> 128 (ReLU) -> 128 (ReLU) -> 4, parameters in one flat array (row-major, out x in):
W1[128][32], b1[128], W2[128][128], b2[128], W3[4][128], b3[4].  Inputs are standardised
with norm = (x_mean[32], x_std[32], t_mean[4], t_std[4]); the outputs o are standardised
targets; the loss is the mean over samples and outputs of (o - (t - t_mean) / t_std)^2.
Forward pass, loss and the backward pass (chain rule, layer by layer) in numpy FP64; Adam
as published (Kingma and Ba, 2015: bias-corrected first and second moment estimates).
"""
from __future__ import annotations

import numpy as np

SIZES = [("W1", (128, 32)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
         ("W3", (4, 128)), ("b3", (4,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def _split_norm(norm):
    norm = np.asarray(norm, dtype=np.float64)
    return norm[:32], norm[32:64], norm[64:68], norm[68:72]


def forward(params, norm, X):
    """Predictions o * t_std + t_mean, (nsamples, 4)."""
    P = unpack(params)
    xm, xsd, tm, tsd = _split_norm(norm)
    x = (np.asarray(X, dtype=np.float64) - xm) / xsd
    h1 = np.maximum(x @ P["W1"].T + P["b1"], 0.0)
    h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0.0)
    o = h2 @ P["W3"].T + P["b3"]
    return o * tsd + tm


def loss_grad(params, norm, X, T):
    """(loss, gradient as a flat array in the parameter layout)."""
    P = unpack(params)
    xm, xsd, tm, tsd = _split_norm(norm)
    x = (np.asarray(X, dtype=np.float64) - xm) / xsd
    t = (np.asarray(T, dtype=np.float64) - tm) / tsd
    B = x.shape[0]
    a1 = x @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ P["W3"].T + P["b3"]
    r = o - t
    loss = np.mean(r * r)
    do = 2.0 * r / (B * 4)
    g = {"W3": do.T @ h2, "b3": do.sum(axis=0)}
    d2 = (do @ P["W3"]) * (a2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"]) * (a1 > 0)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SIZES])


def adam_step(params, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Returns (params, m, v) after one Adam step."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(rng, scale=1.0):
    """He-style random initialisation (for tests and training)."""
    parts = []
    for name, shape in SIZES:
        if name.startswith("W"):
            parts.append(rng.standard_normal(shape).ravel() * scale * np.sqrt(2.0 / shape[1]))
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts)

"""Learned starting point for Fisher scoring (an addition to the paper's method, whose fits
start from fixed rules): training data, training, and use with a fallback.

The simulation, the fits, the features, the network's training and inference and the
learned start with its fallback, the fields' variances and the training targets run in
the library's CUDA kernels through the C ABI.  This module orders those calls; PyTorch
provides device memory and the seeded random inputs (normal variates, random index pairs,
sample permutations).

Fields are isotropic Matern fields at one shared set of n locations (maxmin order and
ordered-neighbour array supplied by the caller), X = 1 (beta = 0):

  * priors (one draw per field): sigma2, rho, nu, tau2 log-uniform on [0.5, 2],
    [0.02, 0.3], [0.5, 2.5], [0.001, 0.2];
  * simulation: the sequential Vecchia draw of the NNarray (vecchia_fields_simulate);
  * targets: the plain method's optimum, a Fisher-scoring fit from the default start
    (var y, 0.1, 1, 0.1) (vecchia_fields_fit), as (log(sigma2 / var y), log rho, log nu,
    log tau2) clamped to TARGET_RANGE; fields whose fit does not converge are left out of
    the training set;
  * features: 32 log-spaced lag bins on [0.005, 0.5] of the empirical semivariogram over
    the NNarray pairs and 2^20 random pairs (vecchia_fields_variogram);
  * network and training: 32 -> 128 -> 128 -> 4 (vecchia_mlp_*), Adam on the mean squared
    error of the standardised targets, minibatches from a random permutation per epoch;
  * use: vecchia_fields_warm_start, which keeps the predicted start only where it is
    finite and its loglik is not below the default start's.
"""
from __future__ import annotations

import os
import time
from dataclasses import dataclass

import numpy as np

from . import (MATERN_ISO, MLP_NPARAMS, vecchia_fields_fit, vecchia_fields_moments,
               vecchia_fields_simulate, vecchia_fields_variogram, vecchia_fields_warm_start,
               vecchia_mlp_adam_step, vecchia_mlp_column_moments, vecchia_mlp_forward,
               vecchia_mlp_grad, vecchia_mlp_targets, vecchia_mlp_theta)

PRIORS = {"sigma2": (0.5, 2.0), "rho": (0.02, 0.3), "nu": (0.5, 2.5), "tau2": (0.001, 0.2)}
NBINS, LAG_LO, LAG_HI = 32, 0.005, 0.5
NRAND = 2 ** 20


@dataclass
class Geometry:
    """Shared locations of a set of fields, on the device."""
    locs: object      # (n, 2) float64
    NN: object        # (n, m+1) int32
    X: object         # (n, 1) float64 ones
    edges2: object    # (NBINS + 1) float64 squared lag edges
    rand_pairs: object  # (NRAND, 2) int32 (the bits of uint32 words)

    @property
    def n(self):
        return self.locs.shape[0]

    @property
    def m(self):
        return self.NN.shape[1] - 1


def make_geometry(locs, NN, device="cuda:0", seed: int = 0) -> Geometry:
    import torch
    dev = torch.device(device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    words = torch.randint(-2 ** 31, 2 ** 31, (NRAND, 2), generator=g, dtype=torch.int64)
    return Geometry(
        locs=torch.as_tensor(np.ascontiguousarray(locs), dtype=torch.float64, device=dev),
        NN=torch.as_tensor(np.ascontiguousarray(NN), dtype=torch.int32, device=dev),
        X=torch.ones(len(locs), 1, dtype=torch.float64, device=dev),
        edges2=torch.as_tensor(np.geomspace(LAG_LO, LAG_HI, NBINS + 1) ** 2, dtype=torch.float64,
                               device=dev),
        rand_pairs=words.to(torch.int32).to(dev))


def sample_priors(rng: np.random.Generator, nfields: int) -> np.ndarray:
    cols = [np.exp(rng.uniform(np.log(lo), np.log(hi), nfields)) for lo, hi in PRIORS.values()]
    return np.column_stack(cols)


def default_start(Y):
    """(var y, 0.1, 1, 0.1) per field, on the device (FP64 variance of each row)."""
    import torch
    _, var = vecchia_fields_moments(Y)
    s = torch.empty(Y.shape[0], 4, dtype=torch.float64, device=Y.device)
    s[:, 0] = var
    s[:, 1] = 0.1
    s[:, 2] = 1.0
    s[:, 3] = 0.1
    return s


def simulate_fields(geom: Geometry, theta: np.ndarray, seed: int):
    import torch
    dev = geom.locs.device
    g = torch.Generator(device=dev).manual_seed(seed)
    z = torch.randn(len(theta), geom.n, generator=g, dtype=torch.float64, device=dev)
    th = torch.as_tensor(theta, dtype=torch.float64, device=dev)
    Y, st = vecchia_fields_simulate(geom.locs, geom.NN, th, MATERN_ISO, z)
    return Y, st


# Training targets are clamped to these ranges of (sigma2 / var y, rho, nu, tau2): a fit can
# converge with the nugget driven towards 0 (the likelihood is flat there), and such targets
# (log tau2 of -50 and below) would dominate the squared-error loss.
TARGET_RANGE = ((1e-2, 1e2), (1e-4, 1e1), (0.05, 20.0), (1e-6, 1e1))


def targets_from_fit(theta_hat, Y):
    """(log(sigma2 / var y), log rho, log nu, log tau2), clamped to TARGET_RANGE, float32."""
    _, var = vecchia_fields_moments(Y)
    return vecchia_mlp_targets(theta_hat.contiguous(), var, [r[0] for r in TARGET_RANGE],
                               [r[1] for r in TARGET_RANGE])


def build_training_set(geom: Geometry, nfields: int, seed: int = 1, chunk: int = 4096,
                       prec: str = "mixed", log=print):
    """Simulates and fits nfields fields (chunk at a time); returns (features, targets,
    stats) for the fields whose fit converged."""
    import torch
    rng = np.random.default_rng(seed)
    feats, targs = [], []
    stats = {"fields": 0, "converged": 0, "simulate_s": 0.0, "fit_s": 0.0, "features_s": 0.0}
    for c0 in range(0, nfields, chunk):
        nf = min(chunk, nfields - c0)
        theta = sample_priors(rng, nf)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Y, st = simulate_fields(geom, theta, seed * 1000003 + c0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fit = vecchia_fields_fit(geom.locs, geom.X, geom.NN, Y, MATERN_ISO, default_start(Y),
                                 prec=prec)
        t2 = time.perf_counter()
        f = vecchia_fields_variogram(geom.locs, geom.NN, Y, geom.rand_pairs, geom.edges2)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        ok = torch.as_tensor((fit["status"] == 0) & (st[:, 0].cpu().numpy() == 0), device=Y.device)
        ok &= torch.isfinite(f).all(dim=1)
        feats.append(f[ok])
        targs.append(targets_from_fit(fit["theta"], Y)[ok])
        stats["fields"] += nf
        stats["converged"] += int(ok.sum().item())
        stats["simulate_s"] += t1 - t0
        stats["fit_s"] += t2 - t1
        stats["features_s"] += t3 - t2
        if log:
            log("training set: %d / %d fields, %d kept" % (c0 + nf, nfields, stats["converged"]))
    return torch.cat(feats).contiguous(), torch.cat(targs).contiguous(), stats


LAYERS = [(128, 32), (128, 128), (4, 128)]   # (out, in) of the three layers


def init_params(seed: int):
    """He initialisation (weights N(0, 2 / fan_in), biases 0) in the flat layout."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    parts = []
    for fo, fi in LAYERS:
        parts.append(torch.randn(fo * fi, generator=g, dtype=torch.float64) * np.sqrt(2.0 / fi))
        parts.append(torch.zeros(fo, dtype=torch.float64))
    p = torch.cat(parts).to(torch.float32)
    assert p.numel() == MLP_NPARAMS
    return p


def train(X, T, epochs: int = 60, batch: int = 256, lr: float = 1e-3, seed: int = 2,
          log=print):
    """Adam on the standardised targets, minibatches from a fresh random permutation each
    epoch.  Returns (params, norm, losses): losses["epochs"] holds the last minibatch loss
    of each epoch, losses["initial"] / losses["final"] the loss over the whole training set
    before and after training."""
    import torch
    dev = X.device
    xm, xs = vecchia_mlp_column_moments(X)
    tm, ts = vecchia_mlp_column_moments(T)
    norm = torch.cat([xm, xs, tm, ts]).contiguous()
    P = init_params(seed).to(dev)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed + 1)
    N = X.shape[0]
    step = 0
    losses = {"epochs": [], "initial": float(vecchia_mlp_grad(P, norm, X, T)[1].item())}
    for ep in range(epochs):
        perm = torch.randperm(N, generator=g).to(torch.int32).to(dev)
        for b0 in range(0, N - batch + 1, batch):
            step += 1
            vecchia_mlp_adam_step(P, m, v, step, lr, norm, X, T, index=perm[b0:b0 + batch],
                                  loss=loss)
        losses["epochs"].append(float(loss.item()))
        if log and (ep % 10 == 0 or ep == epochs - 1):
            log("epoch %d: minibatch loss %.4f" % (ep, losses["epochs"][-1]))
    losses["final"] = float(vecchia_mlp_grad(P, norm, X, T)[1].item())
    return P, norm, losses


def save(path: str, params, norm, meta: dict | None = None):
    np.savez(path, params=params.cpu().numpy(), norm=norm.cpu().numpy(),
             meta=np.array(repr(meta or {})))


DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
TRAINED = "warmstart_n4096_m30.npz"   # 50 000 fields of n = 4096, m = 30 (see its .json)


def load(path: str = None, device="cuda:0"):
    """Loads a saved network (default: the one trained by this module's command line on
    50 000 fields of n = 4096, m = 30, shipped in data/)."""
    path = path or os.path.join(DATA, TRAINED)
    import torch
    z = np.load(path)
    return (torch.as_tensor(z["params"], dtype=torch.float32, device=device),
            torch.as_tensor(z["norm"], dtype=torch.float32, device=device))


def predict_theta(params, norm, feats, Y):
    """Predicted parameters (nfields, 4) from features, without the fallback rule (a
    diagnostic; vecchia_fields_warm_start forms its own in a kernel)."""
    pred = vecchia_mlp_forward(params, norm, feats)
    _, var = vecchia_fields_moments(Y)
    return vecchia_mlp_theta(pred.contiguous(), var)


def evaluate(geom: Geometry, params, norm, nfields: int, seed: int = 3, prec: str = "fp64",
             decide_prec: str = "mixed", log=print, detail: bool = False) -> dict:
    """Held-out fields: fits (precision prec) from the default start and from the learned
    start with its fallback rule, each timed as a whole (the learned start's time includes
    the features, the network and its two decision passes, run in decide_prec: they only
    compare two logliks); both must reach the same optimum.  detail=True adds the per-field
    arrays under "fields" (data, optima, logliks, statuses)."""
    import torch
    rng = np.random.default_rng(seed)
    theta = sample_priors(rng, nfields)
    Y, st = simulate_fields(geom, theta, seed * 7919)
    d0 = default_start(Y)
    # warm-up of both paths (kernel loading, graph capture) on the first field
    vecchia_fields_fit(geom.locs, geom.X, geom.NN, Y[:1].contiguous(), MATERN_ISO, d0[:1].contiguous(),
                       prec=prec)
    vecchia_fields_warm_start(params, norm, geom.locs, geom.X, geom.NN, Y[:1].contiguous(),
                              geom.rand_pairs, geom.edges2, d0[:1].contiguous(), prec=decide_prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f_def = vecchia_fields_fit(geom.locs, geom.X, geom.NN, Y, MATERN_ISO, d0, prec=prec)
    t1 = time.perf_counter()
    start, used, _ = vecchia_fields_warm_start(params, norm, geom.locs, geom.X, geom.NN, Y,
                                               geom.rand_pairs, geom.edges2, d0, prec=decide_prec)
    f_ws = vecchia_fields_fit(geom.locs, geom.X, geom.NN, Y, MATERN_ISO, start, prec=prec)
    t2 = time.perf_counter()
    ll_d = f_def["out"][:, 0].cpu().numpy()
    ll_w = f_ws["out"][:, 0].cpu().numpy()
    conv = (f_def["status"] == 0) & (f_ws["status"] == 0)
    rel = np.abs(ll_w - ll_d) / np.maximum(np.abs(ll_d), geom.n)
    same = conv & (rel <= 1e-6)
    used = used.cpu().numpy()
    res = {
        "fields": nfields, "n": geom.n, "m": geom.m, "precision": prec,
        "decision_precision": decide_prec,
        "default": {"seconds": t1 - t0, "mean_iters": float(f_def["iters"].mean()),
                    "mean_passes": float(f_def["evals"].mean()),
                    "max_passes": int(f_def["evals"].max()),
                    "converged": int((f_def["status"] == 0).sum())},
        "learned": {"seconds": t2 - t1, "mean_iters": float(f_ws["iters"].mean()),
                    "mean_passes": float(f_ws["evals"].mean()),
                    "max_passes": int(f_ws["evals"].max()),
                    "converged": int((f_ws["status"] == 0).sum()),
                    "fallback_rate": float(1.0 - used.mean())},
        "both_converged": int(conv.sum()),
        "same_optimum": int(same.sum()),
        "different_optimum_learned_higher": int((conv & ~same & (ll_w > ll_d)).sum()),
        "different_optimum_default_higher": int((conv & ~same & (ll_w < ll_d)).sum()),
        "max_loglik_diff_same": float(rel[same].max()) if same.any() else None,
        "max_loglik_diff": float(rel[conv].max()) if conv.any() else None,
        "loglik_diff_note": "|loglik(learned) - loglik(default)| / max(|loglik|, n); the same "
                            "optimum means a difference <= 1e-6 (the likelihoods can be "
                            "multimodal, and the start decides which maximum is reached)",
        "speedup": (t1 - t0) / (t2 - t1),
    }
    if detail:
        res["fields_detail"] = {
            "Y": Y.cpu().numpy(), "theta_true": theta,
            "theta_default": f_def["theta"].cpu().numpy(), "theta_learned": f_ws["theta"].cpu().numpy(),
            "loglik_default": ll_d, "loglik_learned": ll_w, "converged_both": conv, "same": same}
    if log:
        log("held-out: %s" % res)
    return res


def main(argv=None):
    """Command line: build the training set, train, save the network, evaluate.

    python -m paper_2407_02740_gb300.warmstart --fields 50000 --n 4096 --m 30 --out net.npz
    """
    import argparse
    import json
    import sys
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--fields", type=int, default=50000)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--m", type=int, default=30)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--eval-fields", type=int, default=64)
    ap.add_argument("--eval-n", type=int, default=200000)
    ap.add_argument("--out", default=None, help="where to save the trained network")
    ap.add_argument("--report", default=None)
    ap.add_argument("--evaluate-only", action="store_true",
                    help="skip training: evaluate the network in --net (default: the shipped "
                         "one) and add the result to the report under 'evaluation_<fields>'")
    ap.add_argument("--net", default=None)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import workloads   # seeded input generation: maxmin ordering and ordered neighbours

    def geometry(n, m, seed):
        L = np.random.default_rng(seed).uniform(size=(n, 2))
        L = L[workloads.maxmin_order(L)]
        return make_geometry(L, workloads.ordered_nn(L, m), seed=seed)

    if a.evaluate_only:
        P, norm = load(a.net)
        gev = geometry(a.eval_n, a.m, 1006)
        t0 = time.perf_counter()
        ev = evaluate(gev, P, norm, a.eval_fields, seed=1007)
        ev["wall_s"] = time.perf_counter() - t0
        report = {}
        if a.report and os.path.exists(a.report):
            with open(a.report) as f:
                report = json.load(f)
        report["evaluation_%d_fields" % a.eval_fields] = ev
        if a.report:
            with open(a.report, "w") as f:
                json.dump(report, f, indent=1)
        print(json.dumps(ev))
        return 0
    if not a.out:
        ap.error("--out is required unless --evaluate-only is given")

    t0 = time.perf_counter()
    gtr = geometry(a.n, a.m, 1005)
    X, T, stats = build_training_set(gtr, a.fields)
    t1 = time.perf_counter()
    P, norm, losses = train(X, T, epochs=a.epochs)
    t2 = time.perf_counter()
    meta = {"fields": a.fields, "n": a.n, "m": a.m, "epochs": a.epochs, "kept": int(X.shape[0])}
    save(a.out, P, norm, meta)
    gev = geometry(a.eval_n, a.m, 1006)
    ev = evaluate(gev, P, norm, a.eval_fields)
    report = {"training_set": stats, "training_set_s": t1 - t0, "train_s": t2 - t1,
              "initial_loss": losses["initial"], "final_loss": losses["final"],
              "epoch_losses": losses["epochs"], "evaluation": ev, "meta": meta}
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)
    print(json.dumps(report))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())

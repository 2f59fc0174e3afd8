#!/usr/bin/env python
"""Benchmark: Vecchia loglik + gradient + Fisher information throughput (points/s).

One step = one full ``vecchia_loglik_grad_info`` pass (status reset, Matern table, the
per-observation kernel, the reduction + profile kernel) over the n = 100000, m = 30
isotropic Matern workload (p = 3, four parameters, evaluated at the generating
parameters), with the inputs resident in device memory when the timed region starts.
The inputs (~17 MB) fit in L2, so L2 is flushed (a 256 MB write) before every timed step,
outside the timed region.

Reported beside the device-timed value:
  * e2e        -- the same metric through the host-memory entry point
                  (vecchia_loglik_grad_info_host) from pinned host buffers, with the H2D
                  copies of the inputs and the D2H copy of the result inside the timed region;
  * roofline   -- the per-observation kernel against the FP64 ALU peak (its algorithmic
                  FMA count per observation x observations / its CUDA-event duration);
  * cpu_baseline -- the FP64 CPU oracle on the host cores, on a bounded prefix sample.
  * batched    -- 256 independent fields (n from 1000 to 50000, m in {10, 20, 40}): the
                  batched pass as one CUDA-graph replay vs 256 per-dataset calls, and
                  batched Fisher-scoring fits vs 256 sequential device fits;
  * warm_start -- fits of held-out fields (n = 200000) from the default start and from
                  the learned start;
  * nn_search  -- the ordered nearest-neighbour search and the maxmin ordering on the
                  device vs the CPU versions;
  * prediction -- Vecchia prediction at 100000 new sites of the headline field.
  * elevators_like -- the exponential with one range per attribute on an Elevators-like
                  workload (n = 15000, d = 18): passes, fits, the oracle beside them.
  * grouped    -- grouped conditioning (one factorisation per group of ~8 observations)
                  against the plain pass on the same n = 1e5 ordering.
  * swath      -- the 1.2 M-point space-time swath: FP64 and mixed passes, FP64, mixed-
                  then-FP64 and mixed-only fits, the oracle on a prefix beside them.
``--impl reference`` times the CPU oracle itself as the reference arm.
Multi-GPU runs (torchrun) are independent replicas: each rank evaluates its own copy.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Vecchia lik+grad+info points/s at m=30 (FP64 pass)"
UNIT = "points/s"
WORKLOAD = ("isotropic Matern n=100000 in [0,1]^2, m=30 maxmin-ordered nearest earlier "
            "neighbours, p=3 (1, x1, x2), theta=(2.0, 0.05, 1.5, 0.05), y from a sequential "
            "Vecchia draw with m=60")
# FP64 peak of the GB300 derived from unit counts and clocks: each SM sub-partition
# retires one 32-lane FP64 FMA warp-instruction per 64 cycles (2 FMA/clk/SM, measured by
# a microbenchmark: 596 GFMA/s at ~1.96 GHz), 152 SMs, 2070 MHz maximum SM clock.
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# DRAM bytes (read + write) of one launch of the FP64 pass kernel on this workload, from an
# ncu capture of the current kernel (the summary under profiles/ names the command); set to
# None whenever the kernel changes until it is captured again.
TRAFFIC_BYTES = 17329664 + 0
TRAFFIC_NOTE = "dram__bytes_read.sum + dram__bytes_write.sum, profiles/k_pass_matern_n100000_m30.md"


def algorithmic_fma_per_point(K: int, p: int, q: int) -> float:
    """Cholesky + forward solves of y, X + last-row derivative terms, covariance
    evaluations excluded: (K^3-K)/6 + (2+p)K(K-1)/2 + q(K^2 + K(K-1)/2) + q(1+p)K + q(q+1)K/2."""
    return ((K ** 3 - K) / 6 + (2 + p) * K * (K - 1) / 2 + q * (K * K + K * (K - 1) / 2)
            + q * (1 + p) * K + q * (q + 1) * K / 2)


def covariance_fma_per_point(K: int, covfun: int, d: int) -> float:
    """FP64 work of the covariance and derivative entries as implemented: per off-diagonal
    pair, the squared distance (2d + 1 ops) twice; for the Matern table the two table-
    variable subtractions and the FP64 part of three polynomials (3 FMAs each; the rest of
    each polynomial runs in FP32); for the exponential the square root, exponential and
    division (~35 ops)."""
    pairs = K * (K - 1) / 2
    if covfun == 1:
        return pairs * (2 * (2 * d + 1) + 2 + 3 * 3)
    return pairs * (2 * d + 1 + 35)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thr = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thr = threading.Thread(target=self._read, daemon=True)
        self.thr.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thr:
            self.thr.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(x: float, ws: int) -> float:
    """The largest value of x over the ranks (the slowest replica's time); x itself at N = 1."""
    if ws <= 1:
        return float(x)
    import torch
    tt = torch.tensor([float(x)], dtype=torch.float64)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(ws: int, units_per_rank: int, steps: int, total_s: float) -> float:
    """Whole-job units per second: every rank processes units_per_rank units per step, and
    the job takes the slowest rank's time."""
    return ws * units_per_rank * steps / total_s


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload():
    import workloads
    return workloads.cfg_matern_100k()


def cpu_oracle_rate(w, target_s: float = 12.0, nthreads: int = 0):
    """Times the oracle on a prefix of the workload (all host cores unless nthreads > 0);
    the prefix is sized from a short calibration run to take about target_s seconds."""
    import oracle
    oracle.build()
    th = w.theta_true
    n0 = min(w.n, 3000)
    t0 = time.perf_counter()
    oracle.loglik_grad_info(w.locs[:n0], w.y[:n0], w.X[:n0], w.NN[:n0], th, w.covfun,
                            nthreads=nthreads)
    rate0 = n0 / (time.perf_counter() - t0)
    ns = int(min(w.n, max(n0, rate0 * target_s)))
    t0 = time.perf_counter()
    oracle.loglik_grad_info(w.locs[:ns], w.y[:ns], w.X[:ns], w.NN[:ns], th, w.covfun,
                            nthreads=nthreads)
    dt = time.perf_counter() - t0
    cores = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    return ns / dt, ns, dt, cores


def tuned_table_placement(handle, m: int, prec: int, batched: bool = False):
    """The Matern table placement ("shared" / "global") the handle's autotuning record chose
    for (m, precision), read from its saved records."""
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.json")
        handle.autotune_save(path)
        recs = json.load(open(path))
    want = prec + (2 if batched else 0)
    for r in recs:
        if r["m"] == m and r["prec"] == want:
            return {1: "shared", 0: "global"}.get(r.get("tab", -1), "planner")
    return None


def run_batched(vg, torch, dev, stream, steps: int, warmup: int, flush, local: int) -> dict:
    """The 256-dataset batch (Matern fields, n log-uniform in [1000, 50000], m in
    {10, 20, 40}, per-dataset parameters, X = 1): the batched pass as one CUDA-graph
    replay of a batch plan (mapping from the batched autotuner) against 256 per-dataset
    pass calls, the mixed-precision batched pass, and batched Fisher-scoring fits against
    256 sequential single-dataset device fits.  L2 is flushed before every timed step."""
    import workloads
    t_gen = time.perf_counter()
    bw = workloads.cfg_batch()
    t_gen = time.perf_counter() - t_gen
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    locs, y, X, NN = (t(bw.locs, torch.float64), t(bw.y, torch.float64), t(bw.X, torch.float64),
                      t(bw.NN, torch.int32))
    th, th0 = t(bw.theta_true, torch.float64), t(bw.theta_start, torch.float64)
    nb, q, p = bw.nbatch, 4, 1
    ntot = int(bw.offsets[-1])
    nout = 1 + q + q * q + p
    hb = vg.Handle(local)
    tune = vg.vecchia_batch_autotune(locs, y, X, NN, bw.offsets, bw.m, th, bw.covfun, reps=2,
                                     stream=stream, handle=hb)
    vg.vecchia_batch_autotune(locs, y, X, NN, bw.offsets, bw.m, th, bw.covfun, prec="mixed",
                              reps=2, stream=stream, handle=hb)
    btab = tuned_table_placement(hb, int(max(bw.m)), 0, batched=True)

    def graph_of(plan, cp, out, st):
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            plan.run(locs, y, X, NN, cp, out, st)
        torch.cuda.current_stream(dev).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.run(locs, y, X, NN, cp, out, st)
        return g

    def time_steps(fn, k):
        ms = []
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    res = {}
    for prec in ("fp64", "mixed"):
        plan = vg.BatchPlan(bw.offsets, bw.m, 2, p, bw.covfun, prec=prec, handle=hb, device=local)
        out = torch.empty(nb, nout, dtype=torch.float64, device=dev)
        st = torch.empty(nb, 2, dtype=torch.int64, device=dev)
        g = graph_of(plan, th, out, st)
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize()
        ms = time_steps(g.replay, steps)
        res[prec] = {"out": out.clone(), "status": st.cpu().numpy(), "ms": ms,
                     "mapping": plan.mapping()}
        plan.close()
    if np.any(res["fp64"]["status"][:, 0] != 0):
        raise RuntimeError("batched pass failed: %s" % res["fp64"]["status"][:, 0])

    # the same work as 256 separate pass calls (planned mapping per dataset), one stream
    hs = vg.Handle(local)
    nn_off = np.concatenate([[0], np.cumsum(np.diff(bw.offsets) * (bw.m.astype(np.int64) + 1))])
    views = []
    for b in range(nb):
        s0, e0 = int(bw.offsets[b]), int(bw.offsets[b + 1])
        views.append((locs[s0:e0], y[s0:e0], X[s0:e0],
                      NN[int(nn_off[b]):int(nn_off[b + 1])].view(e0 - s0, int(bw.m[b]) + 1)))
    outs = torch.empty(nb, nout, dtype=torch.float64, device=dev)
    sts = torch.empty(nb, 2, dtype=torch.int64, device=dev)

    def per_dataset():
        for b, (a0, a1, a2, a3) in enumerate(views):
            vg.vecchia_loglik_grad_info(a0, a1, a2, a3, th[b], bw.covfun, stream=stream,
                                        out=outs[b], status=sts[b], handle=hs)
    per_dataset()
    torch.cuda.synchronize()
    ms_sep = time_steps(per_dataset, max(3, steps // 5))
    o64 = res["fp64"]["out"].cpu().numpy()
    osep = outs.cpu().numpy()
    omx = res["mixed"]["out"].cpu().numpy()
    nb_n = np.diff(bw.offsets).astype(np.float64)
    ll_rel_sep = float(np.max(np.abs(o64[:, 0] - osep[:, 0]) / np.maximum(np.abs(osep[:, 0]), nb_n)))
    ll_rel_mixed = float(np.max(np.abs(omx[:, 0] - o64[:, 0]) / np.maximum(np.abs(o64[:, 0]), nb_n)))

    # fits: one batched fit (graph) vs the 256 datasets fitted one after another
    bfit_s, bfit = [], None
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bfit = vg.vecchia_batch_fit(locs, y, X, NN, bw.offsets, bw.m, bw.covfun, th0, tol=1e-4,
                                    stream=stream, handle=hb)
        bfit_s.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mfit = vg.vecchia_batch_fit(locs, y, X, NN, bw.offsets, bw.m, bw.covfun, th0, tol=1e-4,
                                prec="mixed", stream=stream, handle=hb)
    mfit_s = time.perf_counter() - t0
    seq_ll = np.empty(nb)
    seq_iters = np.empty(nb, dtype=np.int64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b, (a0, a1, a2, a3) in enumerate(views):
        f = vg.vecchia_fit(a0, a1, a2, a3, bw.covfun, bw.theta_start[b], tol=1e-4, stream=stream,
                           handle=hs)
        seq_ll[b] = f["loglik"]
        seq_iters[b] = f["iters"]
    seq_s = time.perf_counter() - t0
    bll = bfit["out"][:, 0].cpu().numpy()
    mll = mfit["out"][:, 0].cpu().numpy()
    conv = (bfit["status"] == 0)
    both = conv & (mfit["status"] == 0)
    norm = np.maximum(np.abs(bll), np.diff(bw.offsets).astype(np.float64))
    hs.close()
    hb.close()

    flop = float(sum(2 * algorithmic_fma_per_point(int(mb) + 1, p, q) * (bw.offsets[b + 1] - bw.offsets[b])
                     for b, mb in enumerate(bw.m)))
    b_ms = statistics.median(res["fp64"]["ms"])
    return {
        "workload": "256 Matern fields in [0,1]^2, n log-uniform in [1000, 50000] (total %d), "
                    "m in {10, 20, 40}, per-dataset (sigma2, rho, nu, tau2) drawn from the "
                    "stated priors, X = 1, sequential Vecchia draws with m = 40" % ntot,
        "datasets": nb, "points": ntot, "generation_s": t_gen,
        "value": ntot / (b_ms * 1e-3), "unit": UNIT, "dtype": "f64",
        "ms_per_step": b_ms,
        "launch": "one CUDA-graph replay of a batch plan (set-up, table build, one pass launch "
                  "per block-size class, profile)",
        "gpu_launches_per_step": 3 + len(res["fp64"]["mapping"]["classes"]),
        "mapping": {"lanes_per_observation": tune["lanes"], "threads_per_block": tune["threads"],
                    "matern_table": btab, "classes": res["fp64"]["mapping"]["classes"],
                    "source": "vecchia_batch_autotune (per block-size class)"},
        "roofline": {"bound": "alu", "unit": "GFLOP/s", "peak": FP64_PEAK_GFLOPS,
                     "achieved": flop / (b_ms * 1e-3) / 1e9,
                     "frac": flop / (b_ms * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                     "note": "whole replay (tables, pass, profiles) timed"},
        "per_dataset_launches": {"value": ntot / (statistics.median(ms_sep) * 1e-3), "unit": UNIT,
                                 "ms_per_step": statistics.median(ms_sep),
                                 "gpu_launches_per_step": nb * 4,
                                 "max_loglik_rel_diff_vs_batched": ll_rel_sep},
        "speedup_vs_per_dataset": statistics.median(ms_sep) / b_ms,
        "mixed": {"value": ntot / (statistics.median(res["mixed"]["ms"]) * 1e-3), "unit": UNIT,
                  "ms_per_step": statistics.median(res["mixed"]["ms"]),
                  "mapping": res["mixed"]["mapping"],
                  "max_loglik_rel_diff_vs_fp64": ll_rel_mixed},
        "fit": {"tol": 1e-4, "start": "(var y, 0.1, 1.0, 0.1) per dataset",
                "batched_f64_s": bfit_s[1], "batched_f64_first_call_s": bfit_s[0],
                "batched_mixed_s": mfit_s, "sequential_f64_s": seq_s,
                "speedup_batched_vs_sequential": seq_s / bfit_s[1],
                "converged": int(conv.sum()),
                "status_counts": {str(k): int((bfit["status"] == k).sum()) for k in range(4)},
                "max_iters": int(bfit["iters"].max()), "max_passes": int(bfit["evals"].max()),
                "max_loglik_rel_diff_vs_sequential": float(np.max(np.abs(bll - seq_ll) / np.abs(seq_ll))),
                "max_loglik_diff_mixed_vs_f64": float(np.max(np.abs(mll - bll)[both] / norm[both]))
                if np.any(both) else None,
                "loglik_diff_note": "over datasets where both fits converged, |difference| / "
                                    "max(|loglik|, n) (a field's loglik can be near 0)",
                "sequential_iters_equal": bool(np.array_equal(seq_iters, bfit["iters"]))},
    }


def run_warm_start(torch, dev, local: int, nfields: int = 64) -> dict:
    """The learned start (the network shipped with the package, trained by its own kernels on
    50 000 simulated-and-fitted fields of n = 4096) on held-out fields of n = 200 000,
    m = 30: Fisher-scoring passes and wall time from the default start and from the
    learned start with its fallback rule, and the agreement of the optima."""
    import workloads
    from paper_2407_02740_gb300 import warmstart as ws
    L = np.random.default_rng(1006).uniform(size=(200000, 2))
    L = L[workloads.maxmin_order(L)]
    geom = ws.make_geometry(L, workloads.ordered_nn(L, 30), device=dev, seed=1006)
    params, norm = ws.load(device=dev)
    res = ws.evaluate(geom, params, norm, nfields=nfields, seed=1007, log=None)
    res["workload"] = ("%d held-out Matern fields at one set of n = 200000 uniform locations, "
                       "m = 30, parameters from the training priors" % nfields)
    return res


def run_nn_search(vg, torch, dev, stream) -> dict:
    """Ordered nearest-neighbour search (the NNarray) on the device against the CPU search
    of the same definition on the host cores: the 100000 maxmin-ordered locations of the
    headline workload (m = 30) and 1000000 uniform locations in random order (m = 30);
    the arrays must be identical."""
    import workloads
    res = {}
    for name, n, ordered in (("n100000_maxmin", 100000, True), ("n1000000_random_order", 1000000, False)):
        rng = np.random.default_rng(1002 if ordered else 1008)
        L = rng.uniform(size=(n, 2))
        if ordered:
            L = L[workloads.maxmin_order(L)]
        t0 = time.perf_counter()
        ref = workloads.ordered_nn(L, 30)
        cpu_s = time.perf_counter() - t0
        Ld = torch.as_tensor(L, dtype=torch.float64, device=dev)
        NN = vg.vecchia_ordered_nn(Ld, 30, stream=stream)      # warm-up (scratch allocation)
        ms = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            NN = vg.vecchia_ordered_nn(Ld, 30, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name] = {"n": n, "m": 30, "gpu_ms": statistics.median(ms), "cpu_ms": cpu_s * 1e3,
                     "cpu_threads": os.cpu_count() or 1,
                     "identical": bool(np.array_equal(NN.cpu().numpy(), ref))}
    # the maxmin ordering on the device against the CPU ordering (grid and lazy max-heap,
    # one host thread) on 100000 uniform points and on the 1.2 M-point swath's scaled
    # coordinates; the orders must be identical
    for name, pts in (("maxmin_n100000", np.random.default_rng(1002).uniform(size=(100000, 2))),
                      ("maxmin_swath_n1200000",
                       workloads.swath_locations(np.random.default_rng(1003)) / np.array([5.0, 5.0, 2.0]))):
        t0 = time.perf_counter()
        ref = workloads.maxmin_order(pts)
        cpu_s = time.perf_counter() - t0
        P = torch.as_tensor(pts, dtype=torch.float64, device=dev)
        vg.vecchia_maxmin_order(P, stream=stream)          # warm-up (scratch allocation)
        ms = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            order = vg.vecchia_maxmin_order(P, stream=stream)
            ms.append((time.perf_counter() - t0) * 1e3)
        res[name] = {"n": int(pts.shape[0]), "d": int(pts.shape[1]), "gpu_ms": statistics.median(ms),
                     "cpu_ms": cpu_s * 1e3, "cpu_threads": 1,
                     "identical": bool(np.array_equal(order.cpu().numpy(), ref)),
                     "timing": "wall time around the call (it synchronises), median of 3"}
    return res


def run_prediction(vg, torch, dev, stream, w) -> dict:
    """Vecchia prediction on the headline field (n = 1e5, m = 30, Matern) at 100 000 new
    uniform sites: the neighbour search for the queries and the prediction, each timed with
    CUDA events (median of 3), against the CPU oracle on a sample of targets."""
    import oracle
    from oracle import predict as op
    rng = np.random.default_rng(1009)
    npred = 100000
    Lp = rng.uniform(size=(npred, 2))
    Xp = np.column_stack([np.ones(npred), Lp])
    beta = np.array([1.0, 0.5, -0.5])
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    locs, y, X, th = t(w.locs), t(w.y), t(w.X), t(w.theta_true)
    dLp, dXp, dbeta = t(Lp), t(Xp), t(beta)
    NN = vg.vecchia_nearest(locs, dLp, 30, stream=stream)
    vg.vecchia_predict(locs, y, X, dbeta, dLp, dXp, NN, th, w.covfun, stream=stream)
    nn_ms, pr_ms = [], []
    for _ in range(3):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        NN = vg.vecchia_nearest(locs, dLp, 30, stream=stream)
        e1.record(stream)
        mean, var, st = vg.vecchia_predict(locs, y, X, dbeta, dLp, dXp, NN, th, w.covfun,
                                           stream=stream)
        e2.record(stream)
        e2.synchronize()
        nn_ms.append(e0.elapsed_time(e1))
        pr_ms.append(e1.elapsed_time(e2))
    oracle.build()
    sel = np.arange(0, npred, 100)
    t0 = time.perf_counter()
    mo, vo = op.predict(w.locs, w.y, w.X, beta, Lp[sel], Xp[sel], NN.cpu().numpy()[sel],
                        w.theta_true, w.covfun)
    cpu_s = time.perf_counter() - t0
    mg, vgv = mean.cpu().numpy()[sel], var.cpu().numpy()[sel]
    return {"targets": npred, "m": 30, "status": int(st[0]),
            "nearest_ms": statistics.median(nn_ms), "predict_ms": statistics.median(pr_ms),
            "value": npred / (statistics.median(pr_ms) * 1e-3), "unit": "targets/s",
            "cpu_oracle": {"value": len(sel) / cpu_s, "unit": "targets/s",
                           "sample": "%d targets (every 100th)" % len(sel),
                           "kind": "oracle (numpy dense solve per target)"},
            "max_rel_diff_vs_oracle": {"mean": float(np.max(np.abs(mg - mo) / np.maximum(np.abs(mo), 1e-300))),
                                       "var": float(np.max(np.abs(vgv - vo) / vo))}}


def run_elevators(vg, torch, dev, stream) -> dict:
    """The Elevators-like workload (n = 15000, 18 attributes as locations, exponential with
    one range per attribute, q = 20, X = 1) at m = 10 and m = 30: the FP64 and mixed passes
    in their autotuned mappings (CUDA events, median of 5, inputs resident), the FP64 pass
    against the FP64 peak (algorithmic FMAs as for the headline, q = 20), Fisher-scoring
    fits from the start values (FP64, and mixed then FP64; tol 1e-4, wall time of the
    device fit), and the oracle's pass on the host cores.  The paper's fit times for
    Elevators on its A40 (3.469 s at m = 10, 6.905 s at m = 30) are context."""
    import oracle
    import workloads
    oracle.build()
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    res = {}
    for m, paper_s in ((10, 3.469), (30, 6.905)):
        w = workloads.cfg_elevators_like(m=m)
        q = w.theta_true.size
        locs, y, X, NN, th = t(w.locs), t(w.y), t(w.X), t(w.NN, torch.int32), t(w.theta_true)
        r = {"n": w.n, "d": w.d, "m": m, "q": q}
        for prec in ("fp64", "mixed"):
            h = vg.Handle(0)
            tune = vg.vecchia_autotune(locs, y, X, NN, th, w.covfun, prec=prec, stream=stream, handle=h)
            out, st = vg.vecchia_loglik_grad_info(locs, y, X, NN, th, w.covfun, prec=prec,
                                                  stream=stream, handle=h)
            ms = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vg.vecchia_loglik_grad_info(locs, y, X, NN, th, w.covfun, prec=prec, stream=stream,
                                            out=out, status=st, handle=h)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            r[prec] = {"pass_ms": statistics.median(ms), "points_per_s": w.n / (statistics.median(ms) * 1e-3),
                       "lanes": tune["lanes"], "threads": tune["threads"], "status": int(st[0].item())}
            if prec == "fp64":
                g = vg.unpack(out, q, w.p)
            h.close()
        Kp = (w.NN >= 0).sum(axis=1)
        flop = float(sum(2 * algorithmic_fma_per_point(int(k), w.p, q) for k in Kp))
        r["roofline_fp64_pass"] = {"bound": "alu", "achieved": flop / (r["fp64"]["pass_ms"] * 1e-3) / 1e9,
                                   "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                                   "frac": flop / (r["fp64"]["pass_ms"] * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                                   "note": "pass call (setup, pass kernel, profile) duration; "
                                           "covariance evaluations not counted"}
        for prec in ("fp64", "mixed"):
            h = vg.Handle(0)
            vg.vecchia_fit(locs, y, X, NN, w.covfun, w.theta_start, tol=1e-4, prec=prec,
                           stream=stream, handle=h)                 # graph capture, tuning
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            f = vg.vecchia_fit(locs, y, X, NN, w.covfun, w.theta_start, tol=1e-4, prec=prec,
                               stream=stream, handle=h)
            torch.cuda.synchronize()
            r["fit_" + prec] = {"s": time.perf_counter() - t0, "iters": int(f["iters"]),
                                "evals": int(f["evals"]), "status": vg.FIT_STATUS.get(int(f["status"])),
                                "loglik": float(f["loglik"])}
            h.close()
        r["fit_paper_a40_s"] = paper_s
        t0 = time.perf_counter()
        o = oracle.loglik_grad_info(w.locs, w.y, w.X, w.NN, w.theta_true, w.covfun)
        cpu_s = time.perf_counter() - t0
        r["cpu_oracle"] = {"points_per_s": w.n / cpu_s, "cores": os.cpu_count() or 1,
                           "kind": "oracle", "sample": "one full pass (n = %d)" % w.n}
        r["rel_diff_vs_oracle"] = {"loglik": abs(g["loglik"] - o["loglik"]) / abs(o["loglik"]),
                                   "grad": float(np.linalg.norm(g["grad"] - o["grad"]) /
                                                 max(np.linalg.norm(o["grad"]), np.sqrt(np.trace(o["info"]))))}
        res["m%d" % m] = r
    return res


def run_grouped(vg, torch, dev, stream) -> dict:
    """Grouped conditioning on an n = 1e5 Matern field (the headline's parameters) in a
    grouped ordering (spatially compact groups of about 8 points, at most 12, ordered by the
    maxmin order of their centroids), m = 30: the grouped pass (one Cholesky per group, FP64 and
    mixed; three launch classes by block size; the fastest of six lane/thread mappings)
    against the plain pass (autotuned) with m = 30 and with m = 45 (about the grouped
    conditioning size) on the
    same ordering and NNarray, CUDA events, median of 5, inputs resident."""
    import workloads
    th = np.array([2.0, 0.05, 1.5, 0.05])
    w, goff = workloads.grouped_field(100000, 1, th, 30, 8, p=3, seed=1011, m_sim=30,
                                      beta=[1.0, 0.5, -0.5], gmax=12)
    off, idx, nm, kmax = vg.vecchia_group_blocks(w.NN, goff)
    gorder, coff, ckmax = vg.vecchia_group_classes(off, 3)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    locs, y, X, NN, dth = t(w.locs), t(w.y), t(w.X), t(w.NN, torch.int32), t(th)
    doff, didx, dnm = t(off, torch.int64), t(idx, torch.int32), t(nm, torch.int32)
    classes = (t(gorder, torch.int32), coff, ckmax)
    # the plain pass at a conditioning size like the grouped one's (each member conditions
    # on about 45 earlier observations: its group's U and the earlier members)
    NN45 = t(workloads.ordered_nn(w.locs, 45), torch.int32)

    def timed(fn):
        fn()
        ms = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out, st = fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms), out, st

    res = {"n": w.n, "m": 30, "groups": len(goff) - 1, "mean_group": float(np.mean(nm)),
           "mean_block": float(np.mean(np.diff(off))), "largest_block": int(kmax),
           "launch_classes": {"groups": np.diff(coff).tolist(), "largest_block": ckmax.tolist()}}
    for prec in ("fp64", "mixed"):
        # the grouped pass in each mapping (lanes per group x threads x members formed
        # together, 0 = the planner's choice); the fastest is kept
        best = None
        for lanes, threads in ((8, 64), (8, 128), (16, 128), (16, 256), (32, 128), (32, 256)):
            for chunk in (0, 2, 8):
                hg = vg.Handle(0)
                hg.set_lanes(lanes)
                hg.set_block_threads(threads)
                hg.set_group_chunk(chunk)
                try:
                    ms_g, out_g, st_g = timed(lambda: vg.vecchia_grouped_loglik_grad_info(
                        locs, y, X, doff, didx, dnm, kmax, dth, w.covfun, prec=prec, stream=stream,
                        handle=hg, classes=classes))
                except vg.VecchiaError:
                    hg.close()
                    continue
                hg.close()
                if best is None or ms_g < best[0]:
                    best = (ms_g, out_g, st_g, lanes, threads, chunk)
        ms_g, out_g, st_g, lanes_g, threads_g, chunk_g = best
        hp = vg.Handle(0)
        vg.vecchia_autotune(locs, y, X, NN, dth, w.covfun, prec=prec, stream=stream, handle=hp)
        ms_p, out_p, st_p = timed(lambda: vg.vecchia_loglik_grad_info(
            locs, y, X, NN, dth, w.covfun, prec=prec, stream=stream, handle=hp))
        hp.close()
        h45 = vg.Handle(0)
        vg.vecchia_autotune(locs, y, X, NN45, dth, w.covfun, prec=prec, stream=stream, handle=h45)
        ms_45, out_45, _ = timed(lambda: vg.vecchia_loglik_grad_info(
            locs, y, X, NN45, dth, w.covfun, prec=prec, stream=stream, handle=h45))
        h45.close()
        res[prec] = {"grouped_ms": ms_g, "grouped_points_per_s": w.n / (ms_g * 1e-3),
                     "plain_m45_ms": ms_45, "loglik_plain_m45": float(out_45[0].item()),
                     "grouped_mapping": {"lanes": lanes_g, "threads": threads_g,
                                         "members_together": chunk_g or "planner (up to 4)"},
                     "plain_ms": ms_p, "plain_points_per_s": w.n / (ms_p * 1e-3),
                     "status": [int(st_g[0].item()), int(st_p[0].item())],
                     "loglik_grouped": float(out_g[0].item()), "loglik_plain": float(out_p[0].item())}
    return res


def mixed_fma_split(K: int, p: int, q: int):
    """The algorithmic FMAs of one observation (algorithmic_fma_per_point) split by the
    precision the mixed path does them in: FP64 the pivots' diagonal updates (K(K-1)/2) and
    the per-observation dot products (q(1+p)K + q(q+1)K/2); FP32 the rest."""
    total = algorithmic_fma_per_point(K, p, q)
    f64 = K * (K - 1) / 2 + q * (1 + p) * K + q * (q + 1) * K / 2
    return total - f64, f64


def run_swath(vg, torch, dev, stream, steps: int, warmup: int, flush) -> dict:
    """The satellite-like space-time swath (stands in for the paper's Jason-3 + time data,
    Table 2): n = 1 200 000 points in (lon, lat, time), 16 time slices x 8 swath bands x
    9375, space-time exponential (sigma2 1, spatial range 5 degrees, temporal range 2
    slices, tau2 0.1), X = [1, lat], y from the sequential Vecchia draw with m = 40, m = 30.
    The FP64 and the mixed pass at the generating parameters (inputs 207 MB, larger than
    L2), Fisher-scoring fits from the stated start in FP64, mixed-then-FP64 and mixed only,
    and the FP64 oracle on a prefix of the observations beside them (throughput and the
    FP64 pass's error on the same prefix)."""
    import oracle
    import workloads
    t_gen = time.perf_counter()
    w = workloads.cfg_swath_1m2()
    t_gen = time.perf_counter() - t_gen
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    locs, y, X, NN = (t(w.locs, torch.float64), t(w.y, torch.float64), t(w.X, torch.float64),
                      t(w.NN, torch.int32))
    th = t(w.theta_true, torch.float64)
    q, K = 4, w.m + 1
    res = {"workload": "space-time swath n=%d (16 slices x 8 bands x 9375), exponential "
                       "space-time (1, 5, 2, 0.1), X=[1, lat], m=%d, sequential draw m=40"
                       % (w.n, w.m), "n": w.n, "m": w.m, "p": w.p, "generation_s": t_gen}
    outs = {}
    for prec in ("fp64", "mixed"):
        h = vg.Handle(0)
        h.set_timing(True)
        tune = vg.vecchia_autotune(locs, y, X, NN, th, w.covfun, prec=prec, stream=stream, handle=h)
        out = torch.empty(1 + q + q * q + w.p, dtype=torch.float64, device=dev)
        st = torch.empty(2, dtype=torch.int64, device=dev)
        for _ in range(warmup):
            vg.vecchia_loglik_grad_info(locs, y, X, NN, th, w.covfun, prec=prec, stream=stream,
                                        out=out, status=st, handle=h)
        torch.cuda.synchronize()
        ms, kms = [], []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vg.vecchia_loglik_grad_info(locs, y, X, NN, th, w.covfun, prec=prec, stream=stream,
                                        out=out, status=st, handle=h)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kms.append(h.last_timing()["pass"])
        h.close()
        if int(st[0].item()) != 0:
            raise RuntimeError("swath %s pass failed: %s" % (prec, st.cpu().numpy()))
        outs[prec] = vg.unpack(out, q, w.p)
        step_ms = statistics.median(ms)
        kern = statistics.median(kms)
        flop = 2 * algorithmic_fma_per_point(K, w.p, q) * w.n
        res[prec] = {"value": w.n / (step_ms * 1e-3), "unit": UNIT, "ms_per_step": step_ms,
                     "kernel_ms": kern, "mapping": {"lanes": tune["lanes"], "threads": tune["threads"]},
                     "algorithmic_gflops": flop / (kern * 1e-3) / 1e9}
    r64, rmx = outs["fp64"], outs["mixed"]
    gs = max(float(np.linalg.norm(r64["grad"])), float(np.sqrt(np.trace(r64["info"]))))
    res["mixed"]["vs_fp64_pass"] = {
        "loglik_rel": abs(rmx["loglik"] - r64["loglik"]) / abs(r64["loglik"]),
        "grad_rel": float(np.linalg.norm(rmx["grad"] - r64["grad"])) / gs,
        "info_rel": float(np.linalg.norm(rmx["info"] - r64["info"]) / np.linalg.norm(r64["info"]))}
    # fits from the stated start; the first FP64 call also builds the iteration graph
    fits = {}
    h = vg.Handle(0)
    for name, prec in (("fp64_first_call", "fp64"), ("fp64", "fp64"), ("mixed_then_fp64", "mixed"),
                       ("mixed_only", "mixed_only")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = vg.vecchia_fit(locs, y, X, NN, w.covfun, w.theta_start, tol=1e-4, prec=prec,
                           stream=stream, handle=h)
        fits[name] = {"seconds": time.perf_counter() - t0, "iters": f["iters"],
                      "passes": f["evals"], "status": f["status"], "loglik": f["loglik"],
                      "theta": [float(v) for v in f["theta"]]}
    h.close()
    ref = np.array(fits["fp64"]["theta"])
    for name in ("mixed_then_fp64", "mixed_only"):
        fits[name]["theta_rel_err_vs_fp64_fit"] = [float(v) for v in
                                                   np.abs(np.array(fits[name]["theta"]) - ref) / ref]
        fits[name]["loglik_rel_to_fp64_fit"] = abs(fits[name]["loglik"] - fits["fp64"]["loglik"]) / \
            abs(fits["fp64"]["loglik"])
    res["fit"] = dict(fits, tol=1e-4, start=[float(v) for v in w.theta_start],
                      paper_a40_s={"m10": 10.279, "m30": 23.888,
                                   "note": "Jason-3 + time, n = 960k, Table 2 (context)"})
    # the FP64 oracle on a prefix: its rate on the host cores and the FP64 pass's error there
    rate, ns, dt, cores = cpu_oracle_rate(w, target_s=8.0)
    o = oracle.loglik_grad_info(w.locs[:ns], w.y[:ns], w.X[:ns], w.NN[:ns], w.theta_true, w.covfun)
    out, st = vg.vecchia_loglik_grad_info(locs[:ns], y[:ns], X[:ns], NN[:ns], th, w.covfun,
                                          stream=stream)
    g = vg.unpack(out, q, w.p)
    sc = max(float(np.linalg.norm(o["grad"])), float(np.sqrt(np.trace(o["info"]))))
    res["cpu_oracle"] = {"points_per_s": rate, "cores": cores, "kind": "oracle",
                         "sample": "first %d observations, %.1f s" % (ns, dt),
                         "fp64_pass_rel_err_on_sample": {
                             "loglik": abs(g["loglik"] - o["loglik"]) / abs(o["loglik"]),
                             "grad": float(np.linalg.norm(g["grad"] - o["grad"])) / sc,
                             "info": float(np.linalg.norm(g["info"] - o["info"]) / np.linalg.norm(o["info"]))}}
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload()
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # each step: the oracle on a bounded prefix sized so the whole run stays short
    rate, ns, dt, _ = cpu_oracle_rate(w, target_s=4.0)
    times = []
    for _ in range(args.warmup):
        oracle.loglik_grad_info(w.locs[:ns], w.y[:ns], w.X[:ns], w.NN[:ns], w.theta_true, w.covfun)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.loglik_grad_info(w.locs[:ns], w.y[:ns], w.X[:ns], w.NN[:ns], w.theta_true, w.covfun)
        times.append(time.perf_counter() - t0)
    step_s = statistics.mean(times)
    value = ns / step_s
    sample = "first %d of %d observations (maxmin order) per step, OpenMP over observations" % (ns, w.n)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n": w.n, "m": w.m, "p": w.p,
                       "covfun": "matern_iso", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import paper_2407_02740_gb300 as vg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(vg.LIB_PATH):
        vg.build()
    w = make_workload()
    q = 4
    K = w.m + 1
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa
    locs, y, X = t(w.locs, torch.float64), t(w.y, torch.float64), t(w.X, torch.float64)
    NN, th = t(w.NN, torch.int32), t(w.theta_true, torch.float64)
    h = vg.Handle(local)
    h.set_timing(True)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(1 + q + q * q + w.p, dtype=torch.float64, device=dev)
    st = torch.empty(2, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        vg.vecchia_loglik_grad_info(locs, y, X, NN, th, w.covfun, stream=stream, out=out,
                                    status=st, handle=h)

    # untimed: pick the kernel mapping for this problem (recorded in the handle)
    tune = vg.vecchia_autotune(locs, y, X, NN, th, w.covfun, stream=stream, handle=h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if int(st[0].item()) != 0:
        raise RuntimeError("pass failed with status %s" % st.cpu().numpy())

    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    step_ms, pass_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        pass_ms.append(h.last_timing()["pass"])
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), ws)
    ms_per_step = total_ms / args.steps
    value = job_throughput(ws, w.n, args.steps, total_ms / 1e3)

    # end to end through the host-memory entry point, pinned host buffers
    pin = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory().numpy()  # noqa
    hl, hy, hX = pin(w.locs, torch.float64), pin(w.y, torch.float64), pin(w.X, torch.float64)
    hNN, hth = pin(w.NN, torch.int32), pin(w.theta_true, torch.float64)
    he = vg.Handle(local)
    # the autotuned mapping carried over through the saved records, as a caller would
    with tempfile.TemporaryDirectory() as dtmp:
        tpath = os.path.join(dtmp, "tune.json")
        h.autotune_save(tpath)
        he.autotune_load(tpath)
    for _ in range(2):
        vg.vecchia_loglik_grad_info_host(hl, hy, hX, hNN, hth, w.covfun, handle=he)
    e2e_s = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = vg.vecchia_loglik_grad_info_host(hl, hy, hX, hNN, hth, w.covfun, handle=he)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(sum(e2e_s), ws)
    h2d = hl.nbytes + hy.nbytes + hX.nbytes + hNN.nbytes + hth.nbytes
    d2h = 8 * (1 + q + q * q + w.p) + 16

    # the same pass in mixed precision (FP32 block arithmetic, FP64 sums), same timing rules
    hm = vg.Handle(local)
    hm.set_timing(True)
    outm = torch.empty_like(out)
    stm = torch.empty_like(st)
    tune_m = vg.vecchia_autotune(locs, y, X, NN, th, w.covfun, prec="mixed", stream=stream, handle=hm)
    for _ in range(args.warmup):
        vg.vecchia_loglik_grad_info(locs, y, X, NN, th, w.covfun, prec="mixed", stream=stream,
                                    out=outm, status=stm, handle=hm)
    torch.cuda.synchronize()
    mixed_ms, mixed_pass_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vg.vecchia_loglik_grad_info(locs, y, X, NN, th, w.covfun, prec="mixed", stream=stream,
                                    out=outm, status=stm, handle=hm)
        e1.record(stream)
        e1.synchronize()
        mixed_ms.append(e0.elapsed_time(e1))
        mixed_pass_ms.append(hm.last_timing()["pass"])
    mixed_res = vg.unpack(outm, q, w.p)

    # Fisher-scoring fit from the workload's starting point (tol 1e-4): the first call
    # builds the iteration graph, the second reuses it; both are wall time around the call
    fit_times, fit = [], None
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fit = vg.vecchia_fit(locs, y, X, NN, w.covfun, w.theta_start, tol=1e-4, stream=stream,
                             handle=h)
        fit_times.append(time.perf_counter() - t0)

    mfit_times, mfit = [], None
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mfit = vg.vecchia_fit(locs, y, X, NN, w.covfun, w.theta_start, tol=1e-4, prec="mixed",
                              stream=stream, handle=hm)
        mfit_times.append(time.perf_counter() - t0)
    # a fit that stays in mixed precision to the end: its optimum against the FP64 fit's
    ofit_times, ofit = [], None
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ofit = vg.vecchia_fit(locs, y, X, NN, w.covfun, w.theta_start, tol=1e-4,
                              prec="mixed_only", stream=stream, handle=hm)
        ofit_times.append(time.perf_counter() - t0)

    batched = run_batched(vg, torch, dev, stream, args.steps, args.warmup, flush, local)
    warm = run_warm_start(torch, dev, local)
    nn = run_nn_search(vg, torch, dev, stream)
    pred = run_prediction(vg, torch, dev, stream, w)
    elev = run_elevators(vg, torch, dev, stream)
    grouped = run_grouped(vg, torch, dev, stream)
    swath = run_swath(vg, torch, dev, stream, max(3, args.steps // 2), args.warmup, flush)

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
        return 0

    res = vg.unpack(out, q, w.p)
    gscale = max(float(np.linalg.norm(res["grad"])), float(np.sqrt(np.trace(res["info"]))))
    fma_pt = algorithmic_fma_per_point(K, w.p, q)
    cov_pt = covariance_fma_per_point(K, w.covfun, w.d)
    kern_ms = statistics.mean(pass_ms)
    achieved = 2 * fma_pt * w.n / (kern_ms * 1e-3) / 1e9
    achieved_cov = 2 * (fma_pt + cov_pt) * w.n / (kern_ms * 1e-3) / 1e9
    bytes_pt = 4 * K + 8 * (w.d + 1 + w.p)
    cpu_rate, cpu_n, cpu_s, cpu_cores = cpu_oracle_rate(w)
    cpu1_rate, cpu1_n, cpu1_s, _ = cpu_oracle_rate(w, target_s=6.0, nthreads=1)
    peaks = vg.vecchia_measure_peaks(h)
    f32_pt, f64_pt = mixed_fma_split(K, w.p, q)
    mk_ms = statistics.mean(mixed_pass_ms)
    m_ach32 = 2 * f32_pt * w.n / (mk_ms * 1e-3) / 1e9
    m_ach64 = 2 * f64_pt * w.n / (mk_ms * 1e-3) / 1e9
    th_f64 = np.array(fit["theta"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": w.n, "m": w.m, "p": w.p, "covfun": "matern_iso",
                   "point": "generating parameters", "l2": "flushed (256 MB write) before each step",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "alu", "unit": "GFLOP/s", "achieved": achieved,
                     "peak": FP64_PEAK_GFLOPS, "frac": achieved / FP64_PEAK_GFLOPS,
                     "traffic": TRAFFIC_BYTES, "traffic_note": TRAFFIC_NOTE,
                     "kernel": "k_pass<MATERN, L, double> (per-observation pass)",
                     "kernel_ms": kern_ms, "flop_per_point": 2 * fma_pt,
                     "achieved_incl_covariance": achieved_cov,
                     "frac_incl_covariance": achieved_cov / FP64_PEAK_GFLOPS,
                     "frac_of_measured_fp64_fma_chain": achieved / peaks["fp64_gflops"],
                     "peak_note": "FP64 FMA units: 152 SMs x 2 FMA/clk x 2070 MHz",
                     "hbm_gbs": bytes_pt * w.n / (kern_ms * 1e-3) / 1e9,
                     "hbm_frac_of_measured": bytes_pt * w.n / (kern_ms * 1e-3) / 1e9 / 6785.9},
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": cpu_cores, "kind": "oracle",
                         "sample": "first %d of %d observations, %.1f s" % (cpu_n, w.n, cpu_s),
                         "one_core": {"value": cpu1_rate, "unit": UNIT, "cores": 1,
                                      "sample": "first %d observations, %.1f s" % (cpu1_n, cpu1_s)}},
        "measured_peaks": dict(peaks, source="vecchia_measure_peaks (FMA chains, covariance "
                                             "evaluations as the pass does them, FP64 "
                                             "m8n8k4 tensor-core chains)",
                               fp64_peak_from_unit_counts_gflops=FP64_PEAK_GFLOPS),
        "e2e": {"value": job_throughput(ws, w.n, args.steps, e2e_total), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": args.steps * int(vg.lib().vecchia_kernels_per_pass(w.covfun)),
        "clocks": clocks,
        "mapping": {"lanes_per_observation": tune["lanes"], "threads_per_block": tune["threads"],
                    "matern_table": tuned_table_placement(h, w.m, 0),
                    "source": "vecchia_autotune"},
        "fit": {"precision": "f64", "tol": 1e-4, "start": [float(v) for v in w.theta_start],
                "seconds_first_call": fit_times[0], "seconds": fit_times[1],
                "iters": fit["iters"], "passes": fit["evals"], "status": fit["status"],
                "theta": [float(v) for v in fit["theta"]], "loglik": fit["loglik"]},
        "result": {"loglik": res["loglik"], "grad": [float(v) for v in res["grad"]]},
        "mixed": {"dtype": "f32 block / f64 sums",
                  "value": w.n * args.steps / (sum(mixed_ms) / 1e3), "unit": UNIT,
                  "ms_per_step": sum(mixed_ms) / args.steps,
                  "kernel_ms": statistics.mean(mixed_pass_ms),
                  "mapping": {"lanes_per_observation": tune_m["lanes"],
                              "threads_per_block": tune_m["threads"],
                              "matern_table": tuned_table_placement(hm, w.m, 1)},
                  "vs_fp64_pass": {
                      "loglik_rel": abs(mixed_res["loglik"] - res["loglik"]) / abs(res["loglik"]),
                      "grad_rel": float(np.linalg.norm(mixed_res["grad"] - res["grad"])) / gscale,
                      "info_rel": float(np.linalg.norm(mixed_res["info"] - res["info"])
                                        / np.linalg.norm(res["info"]))},
                  "roofline": {"bound": "alu", "unit": "GFLOP/s", "kernel_ms": mk_ms,
                               "fp32": {"achieved": m_ach32, "peak": peaks["fp32_gflops"],
                                        "frac": m_ach32 / peaks["fp32_gflops"],
                                        "flop_per_point": 2 * f32_pt},
                               "fp64": {"achieved": m_ach64, "peak": FP64_PEAK_GFLOPS,
                                        "frac": m_ach64 / FP64_PEAK_GFLOPS,
                                        "flop_per_point": 2 * f64_pt},
                               "note": "algorithmic FMAs split by the precision the mixed "
                                       "path does them in (FP64: pivot diagonal updates and "
                                       "per-observation dot products); FP32 peak measured "
                                       "by the FMA-chain microbenchmark"},
                  "fit_mixed_only": {"precision": "mixed throughout", "tol": 1e-4,
                                     "seconds_first_call": ofit_times[0], "seconds": ofit_times[1],
                                     "iters": ofit["iters"], "passes": ofit["evals"],
                                     "status": ofit["status"], "loglik": ofit["loglik"],
                                     "loglik_rel_to_f64_fit": abs(ofit["loglik"] - fit["loglik"]) / abs(fit["loglik"]),
                                     "theta": [float(v) for v in ofit["theta"]],
                                     "theta_rel_err_vs_f64_fit": [float(v) for v in
                                                                  np.abs(np.array(ofit["theta"]) - th_f64) / th_f64]},
                  "fit": {"precision": "mixed then f64 polish", "tol": 1e-4,
                          "seconds_first_call": mfit_times[0], "seconds": mfit_times[1],
                          "iters": mfit["iters"], "passes": mfit["evals"],
                          "status": mfit["status"], "loglik": mfit["loglik"],
                          "loglik_rel_to_f64_fit": abs(mfit["loglik"] - fit["loglik"]) / abs(fit["loglik"]),
                          "theta": [float(v) for v in mfit["theta"]]}},
        "batched": batched,
        "warm_start": warm,
        "nn_search": nn,
        "prediction": pred,
        "elevators_like": elev,
        "grouped": grouped,
        "swath": swath,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""Training and evaluation driver of the learned census schedule.

Every computation runs in libtc.so kernels (features, profiled census, sample collection,
normalisation, forward/backward, Adam, inference); this module only allocates device buffers
through PyTorch and calls the C ABI in order:

  1. build R-MAT training graphs (scales 18-22 by default, seeds = scales);
  2. run the plain census with per-vertex SM-cycle profiling (tc_census_profile);
  3. collect (features, log cycles) of the vertices split into CTA work items;
  4. fit the input standardisation and the cycles -> plan-units factor (kappa);
  5. train the 4-32-32-1 network with Adam (tc_costmodel_train);
then tc_graph_attach_costmodel makes TC_SCHED_LEARNED plans use its predictions.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import (TC_ALGO_SUFFIX, TC_SCHED_LEARNED, Graph, tc_census_async, tc_census_grid, tc_census_profile,
               tc_costmodel_create,
               tc_costmodel_fit_norm, tc_costmodel_predict, tc_costmodel_samples, tc_costmodel_train,
               tc_graph_attach_costmodel, tc_graph_features)

PLAIN = {"algo": TC_ALGO_SUFFIX}
LEARNED = {"algo": TC_ALGO_SUFFIX, "schedule": TC_SCHED_LEARNED}


def profile_graph(g: Graph, options=None, stream=None, repeats: int = 2):
    """Per-vertex SM cycles of a plain census (the last of `repeats` runs) as a device tensor."""
    import torch
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    vcost = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    for _ in range(repeats):
        vcost.zero_()
        tc_census_profile(g.handle, out, vcost, stream=stream, options=options or PLAIN)
    torch.cuda.synchronize()
    return vcost


def collect(graphs, options=None, stream=None):
    """Training samples of already-built graphs: (X [count, 4], Y [count], count, kappa)."""
    import torch
    cap = sum(g.n for g in graphs)
    X = torch.empty(max(cap, 1) * 4, dtype=torch.float32, device="cuda")
    Y = torch.empty(max(cap, 1), dtype=torch.float32, device="cuda")
    count, est, cyc = 0, 0.0, 0.0
    for g in graphs:
        feat = torch.empty(g.n * 4, dtype=torch.float32, device="cuda")
        tc_graph_features(g.handle, feat, stream=stream)
        vcost = profile_graph(g, options, stream)
        c, e, y = tc_costmodel_samples(g.handle, vcost, feat, X[count * 4:], Y[count:], cap - count, stream=stream)
        count, est, cyc = count + c, est + e, cyc + y
    return X, Y, count, (est / cyc if cyc > 0 else 1.0)


def train_cost_model(scales=(18, 19, 20, 21, 22), seeds=None, steps: int = 800, lr: float = 3e-3, seed: int = 0,
                     stream=None, options=None):
    """Train on R-MAT graphs (edge factor 16, 20% reciprocated); returns (model handle, info)."""
    import graphgen
    seeds = seeds or scales
    t0 = time.perf_counter()
    graphs = []
    try:
        for sc, sd in zip(scales, seeds):
            n, s, d = graphgen.rmat(sc, 16, 0.2, sd)
            graphs.append(Graph.from_arcs(n, s, d, stream=stream, options=options or PLAIN))
        t1 = time.perf_counter()
        X, Y, count, kappa = collect(graphs, options, stream)
    finally:
        for g in graphs:
            g.close()
    t2 = time.perf_counter()
    model = tc_costmodel_create(seed)
    tc_costmodel_fit_norm(model, X, Y, count, kappa, stream=stream)
    loss0 = tc_costmodel_train(model, X, Y, count, 0, lr, stream=stream) if count else float("nan")
    loss = tc_costmodel_train(model, X, Y, count, steps, lr, stream=stream)
    t3 = time.perf_counter()
    return model, {"samples": count, "kappa": kappa, "loss_initial": loss0, "loss_final": loss, "steps": steps,
                   "scales": list(scales), "seeds": list(seeds), "graph_build_s": t1 - t0, "profile_s": t2 - t1,
                   "train_s": t3 - t2}


def prediction_quality(model, g: Graph, options=None, stream=None):
    """Held-out fit of log(measured cycles) per CTA-item vertex: RMS log error of the model and of
    the plain degree estimate, each after the best constant scale (so only the shape counts)."""
    import torch
    X = torch.empty(g.n * 4, dtype=torch.float32, device="cuda")
    Y = torch.empty(g.n, dtype=torch.float32, device="cuda")
    feat = torch.empty(g.n * 4, dtype=torch.float32, device="cuda")
    tc_graph_features(g.handle, feat, stream=stream)
    vcost = profile_graph(g, options, stream)
    count, _, _ = tc_costmodel_samples(g.handle, vcost, feat, X, Y, g.n, stream=stream)
    pred = torch.empty(max(count, 1), dtype=torch.float32, device="cuda")
    tc_costmodel_predict(model, X, count, pred, stream=stream)
    torch.cuda.synchronize()
    y = Y[:count].double().cpu().numpy()
    lp = np.log(np.maximum(pred[:count].double().cpu().numpy(), 1e-30))
    # plain estimate from the same features: P * (mean degree + ...) is proportional, for these
    # vertices, to deg * (neighbour mean); its log shape is log(deg) + const at fixed graph
    fx = X[:count * 4].view(-1, 4).double().cpu().numpy()
    lplain = np.log(np.expm1(fx[:, 2]))
    def rms(a):
        r = y - a
        r = r - r.mean()
        return float(math.sqrt(np.mean(r * r))) if len(r) else float("nan")
    return {"vertices": count, "rms_log_err_model": rms(lp), "rms_log_err_degree": rms(lplain)}


def census_ms(g: Graph, options, stream_obj, reps: int = 5):
    """Median device time of the census under `options` (CUDA events on the stream)."""
    import statistics
    import torch
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    sh = stream_obj.cuda_stream
    tc_census_async(g.handle, out, stream=sh, options=options)
    stream_obj.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream_obj)
        tc_census_async(g.handle, out, stream=sh, options=options)
        e1.record(stream_obj)
        stream_obj.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), [int(x) & ((1 << 64) - 1) for x in out.cpu().tolist()]


def balance(g: Graph, options, stream=None, reps: int = 3):
    """Work balance of the census under `options` from its per-CTA timestamps (the last of `reps`
    profiled runs; in the triangle form, of the triangle walk): the makespan, the mean CTA busy
    time as a fraction of it, and the tail (the last CTA's end less the median CTA's end)."""
    import torch
    grid = tc_census_grid(options)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    vcost = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    phase = torch.zeros(3 * grid, dtype=torch.int64, device="cuda")
    for _ in range(reps):
        vcost.zero_()
        tc_census_profile(g.handle, out, vcost, phase, stream=stream, options=options)
    torch.cuda.synchronize()
    ph = phase.view(-1, 3).cpu().numpy().astype(np.int64)
    start, end = ph[:, 0], ph[:, 2]
    makespan = float(end.max() - start.min())
    return {"ctas": grid, "makespan_ms": makespan * 1e-6,
            "mean_busy_frac": float((end - start).mean()) / makespan if makespan > 0 else 1.0,
            "tail_ms": float(end.max() - np.median(end)) * 1e-6}


def attach(model, g: Graph, stream=None):
    tc_graph_attach_costmodel(g.handle, model, stream=stream)

"""Benchmark of the GB300 triad census (one JSON line on rank 0).

A step is one full census (Fig. 5) of the scale-20 R-MAT workload: n = 2^20, edge factor
16, a/b/c/d = .57/.19/.19/.05, ids permuted, loops and duplicates dropped, 20% of arcs
reciprocated, seed 2.  `value` is arcs/s with the CSR resident in HBM (device time per
census from CUDA events on the launching stream, L2 flushed by a 512 MB write between
steps, outside the events).  `e2e` is the same metric through the public C ABI from pinned
host arc buffers: graph build (H2D copy, symmetrise, dedupe, relabel, sort) plus census plus
the D2H read of the 16 counts, every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--algo suffix|union] [--impl reference]

--impl reference times the CPU oracle (test infrastructure, single-threaded) on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank runs the same census on its
own GPU (replicas, weak scaling); only the barrier and the max-over-ranks time cross ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "triad-census arcs/sec (bit-exact), learned/batched vs plain; % HBM roofline"
# R-MAT workloads by scale (edge factor 16, a/b/c = .57/.19/.19, ids permuted): scale 20 is the
# bench's default; scale 10 the small parity case; scale 26 the learned-vs-plain comparison
WORKLOADS = {10: dict(name="rmat10_ef16_r15_seed1", scale=10, edge_factor=16, recip=0.15, seed=1),
             20: dict(name="rmat20_ef16_r20_seed2", scale=20, edge_factor=16, recip=0.2, seed=2),
             26: dict(name="rmat26_ef16_r20_seed3", scale=26, edge_factor=16, recip=0.2, seed=3)}
WORKLOAD = dict(WORKLOADS[20])
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_census_rmat20_traffic.txt")
CENSUS_SRC = os.path.join(ROOT, "paper_1209_6308_gb300", "csrc", "census.cu")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--algo", default="suffix", choices=["suffix", "union"])
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-stride", type=int, default=0)
    p.add_argument("--no-batch", action="store_true", help="skip the 4096-graph batched comparison")
    p.add_argument("--autotune-trials", type=int, default=12)
    p.add_argument("--no-learned", action="store_true", help="skip the learned-schedule comparison")
    p.add_argument("--no-serve", action="store_true", help="skip the serving (continuous batching) run")
    p.add_argument("--no-interval", action="store_true", help="skip the interval (windowed stream) census run")
    p.add_argument("--no-census64", action="store_true", help="skip the 64-state census run")
    p.add_argument("--serve-seconds", type=float, default=20.0, help="measured seconds per serving arm")
    p.add_argument("--serve-warmup", type=float, default=5.0, help="unmeasured seconds before them")
    p.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate (requests/s)")
    p.add_argument("--scale", type=int, default=20, choices=sorted(WORKLOADS), help="R-MAT workload scale")
    a = p.parse_args()
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[a.scale])
    return a


def workload():
    import graphgen
    return graphgen.rmat(WORKLOAD["scale"], WORKLOAD["edge_factor"], WORKLOAD["recip"], WORKLOAD["seed"])


_T0 = time.perf_counter()


def log(msg: str) -> None:
    """Progress line on stderr (seconds since start), so a slow section shows where it is."""
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def max_over_ranks(dist, ms: float, device) -> float:
    """The slowest rank's time: the job's time when every rank works on its own replica."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, arcs_per_rank: int, ms: float) -> float:
    """Whole-job arcs/s: every rank censuses its own replica, the job ends with the slowest."""
    return world * arcs_per_rank / (ms * 1e-3)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"tc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
CPU_STRIDE = 256          # cpu_baseline: ~0.2% of the union-walk work, ~30 s on one core
REF_STRIDE = 4096         # reference arm: per-step sample, a few seconds each


def oracle_sample(og, stride, offset):
    """Fig. 5 loop of the CPU oracle over vertices u = offset (mod stride); returns
    (estimated seconds for the full census, sample seconds, work fraction)."""
    sec, _, ws, wt = og.sample(stride, offset)
    frac = ws / wt if wt else 1.0
    return (sec / frac if frac > 0 else float("inf")), sec, frac


def cpu_baseline(n, s, d, arcs, stride):
    import oracle
    og = oracle.SampledGraph(n, s, d)
    full, sec, frac = oracle_sample(og, stride, 0)
    og.close()
    return {"value": arcs / full, "unit": "arcs/s", "cores": 1, "kind": "oracle",
            "sample": (f"single-threaded Fig. 5 oracle over vertices u = 0 (mod {stride}) of the same graph: "
                       f"{sec:.1f} s for {frac * 100:.3f}% of the union-walk work, scaled to the full census")}


def run_reference(args):
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n, s, d = workload()
    arcs = len(s)
    stride = args.cpu_sample_stride or REF_STRIDE
    og = oracle.SampledGraph(n, s, d)
    times, secs, fracs = [], [], []
    for i in range(args.warmup + args.steps):
        full, sec, frac = oracle_sample(og, stride, i % stride)
        if i >= args.warmup:
            times.append(full)
            secs.append(sec)
            fracs.append(frac)
    og.close()
    t = sum(secs) / sum(fracs)         # pooled estimate of the full-census time
    v = arcs / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "arcs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n": n, "arcs": arcs},
            "cpu_baseline": {"value": v, "unit": "arcs/s", "cores": 1, "kind": "oracle",
                             "sample": f"step i: Fig. 5 loop over u = i (mod {stride}); full-census time "
                                       f"estimated as total sample seconds / total work fraction "
                                       f"({sum(fracs) * 100:.3f}% of the union-walk work)"},
            "e2e": {"value": v, "unit": "arcs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def census_code_hash(text: str) -> str:
    """First 16 hex digits of the SHA-256 of census.cu's code: comments, trailing blanks and
    empty lines removed, so that edits of comments alone keep a capture's counters valid."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    code = "\n".join(ln for ln in lines if ln.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def stored_traffic():
    """Per-launch DRAM bytes from the committed ncu summary, if taken on this census.cu code."""
    try:
        kv = dict(line.split(":", 1) for line in open(TRAFFIC_FILE) if ":" in line)
        if kv.get("census_code_sha256_16", "").strip() == census_code_hash(open(CENSUS_SRC).read()):
            return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def batched_comparison(tc, torch, sh, st, trials):
    """4096 Chung-Lu graphs (n log-uniform in [32, 65536], exponent 2.1, mean degree 8, 10%
    reciprocated, seed 4): per-graph launch loop vs one persistent graph-captured launch, default
    and autotuned thresholds.  All three must give identical counts."""
    import graphgen
    specs = graphgen.batch_chung_lu(4096, 32, 65536, 8.0, 2.1, 0.1, 4)
    arcs = int(sum(len(s) for (_, s, _) in specs))
    opts = {"algo": tc.TC_ALGO_SUFFIX}
    gs = [tc.Graph.from_arcs(n, s, d, stream=sh, options=opts) for (n, s, d) in specs]
    handles = [g.handle for g in gs]
    k = len(gs)
    loop_out = torch.zeros(16 * k, dtype=torch.int64, device="cuda")
    batch_out = torch.zeros(16 * k, dtype=torch.int64, device="cuda")

    def timed(fn, reps):
        fn()
        st.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            st.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def loop():
        for i, h in enumerate(handles):
            tc.tc_census_async(h, loop_out[16 * i:16 * i + 16], stream=sh)

    loop_ms = timed(loop, 2)
    b = tc.tc_batch_create(handles, stream=sh, options=opts)
    try:
        batch_ms = timed(lambda: tc.tc_batch_census_async(b, batch_out, stream=sh), 5)
        same_default = bool(torch.equal(batch_out, loop_out))
        t0 = time.perf_counter()
        best, _ = tc.tc_batch_autotune(b, max_trials=trials, stream=sh)
        tune_s = time.perf_counter() - t0
        tuned_ms = timed(lambda: tc.tc_batch_census_async(b, batch_out, stream=sh), 5)
        same_tuned = bool(torch.equal(batch_out, loop_out))
        n_items, n_blocks = tc.tc_batch_stats(b)
    finally:
        tc.tc_batch_destroy(b)
        for g in gs:
            g.close()
    return {"workload": "chunglu4096_n32-65536_g2.1_d8_r10_seed4", "graphs": k, "arcs": arcs,
            "per_graph_loop": {"ms": loop_ms, "arcs_per_s": arcs / (loop_ms * 1e-3), "launches": k},
            "persistent": {"ms": batch_ms, "arcs_per_s": arcs / (batch_ms * 1e-3), "launches": 1},
            "persistent_autotuned": {"ms": tuned_ms, "arcs_per_s": arcs / (tuned_ms * 1e-3), "best": best,
                                     "tuning_s": tune_s, "trials": trials},
            "speedup_vs_loop": loop_ms / min(batch_ms, tuned_ms),
            "items": n_items, "warp_blocks": n_blocks,
            "counts_identical": same_default and same_tuned}


def learned_comparison(tc, g, stream, model, info):
    """Cost model trained on R-MAT scales 18-22 (seeds 18-22) from cycles the plain census
    measures, attached to the bench graph: census time with the plain and the learned schedule
    (identical counts required) and the held-out cost-prediction error of both."""
    from paper_1209_6308_gb300 import learned
    learned.attach(model, g, stream=stream.cuda_stream)
    reps = 5 if g.n <= (1 << 22) else 3
    plain_ms, plain_c = learned.census_ms(g, learned.PLAIN, stream, reps=reps)
    learned_ms, learned_c = learned.census_ms(g, learned.LEARNED, stream, reps=reps)
    q = learned.prediction_quality(model, g, stream=stream.cuda_stream)
    return {"training": info, "plain_ms": plain_ms, "learned_ms": learned_ms,
            "speedup": plain_ms / learned_ms, "counts_identical": plain_c == learned_c,
            "heldout_rms_log_cycle_error": {"model": q["rms_log_err_model"], "degree": q["rms_log_err_degree"],
                                            "vertices": q["vertices"]}}


SERVE_POOL = "pool_chunglu16_n1e3-1e7_d12+rmat16-22_ef16"


def serving_pool():
    """Resident graphs of the serving workload: 16 directed Chung-Lu graphs (n log-uniform in
    [1e3, 1e7], exponent 2.1, mean degree 12, 10% reciprocated, seed 5, graph index i) and R-MAT
    scales 16-22 (edge factor 16, 20% reciprocated, seed 100 + scale)."""
    import graphgen
    sizes = graphgen.loguniform_sizes(16, 1e3, 1e7, 5)
    pool = [(f"chunglu_n{int(n)}", graphgen.chung_lu(int(n), 12.0, 2.1, 0.1, 5, i)) for i, n in enumerate(sizes)]
    pool += [(f"rmat{sc}", graphgen.rmat(sc, 16, 0.2, 100 + sc)) for sc in range(16, 23)]
    return pool


def serve_arm(tc, gs, arcs, census_opts, rate, seconds, warmup, seed):
    """Open-loop Poisson client (rate requests/s, graph i chosen with probability proportional
    to 1/arcs_i so every graph draws the same arc volume) against one server; latency is
    result-complete minus submit on the server's clock.  Every result is checked against the
    graph's standalone census."""
    import threading
    import numpy as np
    rng = np.random.default_rng(seed)
    total = int(rate * (warmup + seconds))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, total))
    w = 1.0 / np.asarray(arcs, dtype=np.float64)
    choice = rng.choice(len(gs), total, p=w / w.sum())
    results, done = [], threading.Event()
    with tc.Server({"quantum_us": 1000, "lanes": 3}, census_opts) as srv:
        ids = [srv.add(g) for g in gs]

        def collector():
            while not done.is_set():
                results.extend(srv.poll(4096, timeout_ms=50))

        th = threading.Thread(target=collector, daemon=True)
        th.start()
        rid_graph, submit_lag = {}, []
        overloaded = False
        t0 = time.perf_counter()
        for k in range(total):
            due = t0 + arrivals[k]
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                if due - now > 2e-3:
                    time.sleep(due - now - 1e-3)
            # an open-loop client against an overloaded server only grows the queue: stop
            if k - len(results) > 20000 or now - t0 > 3.0 * (warmup + seconds):
                overloaded = True
                break
            submit_lag.append(time.perf_counter() - due)
            rid_graph[srv.submit(ids[choice[k]])] = (k, int(choice[k]))
        drained = True
        try:
            srv.drain(120000)
        except tc.TcError:
            drained = False
        finally:
            done.set()
            th.join(timeout=60)
        results.extend(srv.poll(65536))
        stats = srv.stats()
        trace = srv.trace()
    meas = [r for r in results if arrivals[rid_graph[r.id][0]] >= warmup]
    if not meas:
        return {"requests": 0, "completed": len(results), "overloaded": overloaded, "drained": drained,
                "waves": stats["waves"]}, results, rid_graph
    lat = np.array([(r.done_ns - r.submit_ns) * 1e-6 for r in meas])
    t_first = min(r.submit_ns for r in meas)
    t_last = max(r.done_ns for r in meas)
    arcs_done = sum(arcs[rid_graph[r.id][1]] for r in meas)
    return {"requests": len(meas), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "arcs_per_s": arcs_done / ((t_last - t_first) * 1e-9),
            "offered_arcs_per_s": rate * float(np.sum(w / w.sum() * np.asarray(arcs))),
            "achieved_rate": len(meas) / ((t_last - t_first) * 1e-9),
            "gpu_busy_frac": stats["gpu_ms"] * 1e-3 / (time.perf_counter() - t0),
            "waves": stats["waves"], "slices_per_wave": stats["slices"] / max(stats["waves"], 1),
            "mean_waves_per_request": float(np.mean([r.waves for r in results])),
            "submit_lag_p99_ms": float(np.percentile(submit_lag, 99)) * 1e3,
            "errors": int(sum(1 for r in results if r.status != 0)), "completed": len(results),
            "overloaded": overloaded, "drained": drained, "ns_per_unit": stats["ns_per_unit"],
            "wave_gpu_ms": {"p50": float(np.percentile([t["gpu_ms"] for t in trace], 50)),
                            "p99": float(np.percentile([t["gpu_ms"] for t in trace], 99)),
                            "max": float(max(t["gpu_ms"] for t in trace))} if trace else None}, results, rid_graph


def serving_comparison(tc, torch, sh, model, args):
    """Serving workload with the plain and the learned schedule: p50/p99 latency and arcs/s."""
    from paper_1209_6308_gb300 import learned
    t0 = time.perf_counter()
    pool = serving_pool()
    gen_s = time.perf_counter() - t0
    log(f"serving pool generated in {gen_s:.1f}s")
    gs = [tc.Graph.from_arcs(n, s, d, stream=sh, options=learned.PLAIN) for (_, (n, s, d)) in pool]
    arcs = [len(s) for (_, (_, s, _)) in pool]
    want = [g.census(stream=sh, options=learned.PLAIN) for g in gs]
    out = {"workload": SERVE_POOL + f"_poisson{int(args.serve_rate)}_seed5", "graphs": len(gs),
           "pool_arcs": int(sum(arcs)), "rate_per_s": args.serve_rate, "measured_s": args.serve_seconds,
           "warmup_s": args.serve_warmup, "quantum_us": 1000, "lanes": 3, "pool_generation_s": gen_s,
           "selection": "graph i with probability proportional to 1/arcs_i"}
    try:
        arms = [("plain", learned.PLAIN)]
        if model is not None:
            for g in gs:
                learned.attach(model, g, stream=sh)
            arms.append(("learned", learned.LEARNED))
        exact = True
        for name, opts in arms:
            log(f"serving arm {name}")
            m, res, rid_graph = serve_arm(tc, gs, arcs, opts, args.serve_rate, args.serve_seconds,
                                          args.serve_warmup, 5)
            exact &= all(r.census() == want[rid_graph[r.id][1]] for r in res)
            out[name] = m
        out["counts_identical_to_standalone"] = exact
    finally:
        for g in gs:
            g.close()
    return out


def interval_comparison(tc, torch, s, d, n, sh):
    """Interval census (the paper's monitoring use): the bench graph's arcs in a random order at
    uniform times over [0, 1000), a window of 200, a census every 100 from 200 to 1000; each
    census builds the window's graph on the device and counts it (about a fifth of the arcs)."""
    import numpy as np
    rng = np.random.default_rng(7)
    perm = rng.permutation(len(s))
    t = np.sort(rng.integers(0, 1000, len(s))).astype(np.uint64)
    src, dst = s[perm], d[perm]
    times, windows = [], []
    with tc.Stream(n, 200, options={"algo": tc.TC_ALGO_SUFFIX}, stream=sh) as st:
        t0 = time.perf_counter()
        st.push(src, dst, t)
        push_s = time.perf_counter() - t0
        for t_now in range(200, 1001, 100):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, m = st.census(t_now)
            times.append((time.perf_counter() - t1) * 1e3)
            windows.append(m)
    ms = statistics.median(times)
    return {"workload": WORKLOAD["name"] + "_times_uniform1000_window200_every100", "censuses": len(times),
            "arcs_per_window_median": int(statistics.median(windows)), "ms_per_census_median": ms,
            "arcs_per_s": statistics.median(windows) / (ms * 1e-3), "push_s": push_s,
            "note": "per census: window graph build (sort, dedupe, relabel, CSR, tables) + census + D2H of 16 counts"}


def census64_comparison(tc, torch, sh, steps=3):
    """The 64-state census (Sec. 3, Fig. 2) on the R-MAT scale-16 graph (ef16, 20% recip, seed
    16): one thread per linked pair merges the two lists.  Timed with CUDA events around the
    synchronous call (id inversion, census, 512 B D2H); checked by folding the 64 states into
    the 16 classes and comparing with the census of the same graph."""
    import graphgen
    n, s, d = graphgen.rmat(16, 16, 0.2, 16)
    with tc.Graph.from_arcs(n, s, d, stream=sh, options={"algo": tc.TC_ALGO_SUFFIX}) as g:
        info = g.stats()
        c16 = g.census(stream=sh)
        c64 = g.census64(stream=sh)
        times = []
        st = torch.cuda.ExternalStream(sh)
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            c64 = g.census64(stream=sh)
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    table = tc.tc_tricode_table()
    fold = [0] * 16
    for state, k in enumerate(c64):
        fold[int(table[state])] += k
    ms = statistics.median(times)
    # per linked pair both lists are read and each merged entry's original id looked up: 8 B
    # per entry of the two lists (sum over pairs of d_r + d_s = sum_d2); 4 B per CSR entry
    # scanned, and the offsets and id map
    bytes_alg = 8 * info["sum_d2"] + 8 * info["e_sym"] + 16 * (n + 1)
    peak, peak_kind = measured_peak()
    achieved = bytes_alg / (ms * 1e-3) / 1e9
    return {"workload": "rmat16_ef16_r20_seed16", "n": n, "arcs": len(s), "ms": ms,
            "arcs_per_s": len(s) / (ms * 1e-3), "fold_equals_census16": fold == c16,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "k_census64", "bytes_alg_per_launch": bytes_alg}}


def run_gpu(args):
    import torch
    import paper_1209_6308_gb300 as tc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    algo = tc.TC_ALGO_SUFFIX if args.algo == "suffix" else tc.TC_ALGO_UNION
    opts = {"algo": algo}
    log("generating the workload")
    n, s, d = workload()
    arcs = len(s)
    log(f"workload: n={n} arcs={arcs}")
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    g = tc.Graph.from_arcs(n, s, d, stream=sh, options=opts)
    info = g.stats()
    opts_run = opts
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def one_census():
        tc.tc_census_async(g.handle, out, stream=sh, options=opts_run)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            one_census()
    torch.cuda.synchronize()
    log("warm-up done; timing")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                starts[i].record(stream)
                one_census()
                ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = max_over_ranks(dist, statistics.mean(step_ms), "cuda")
    counts = [int(x) & ((1 << 64) - 1) for x in out.cpu().tolist()]
    counts[0] = tc.tc_null_count(n, counts)

    # end to end through the C ABI from pinned host buffers
    if args.e2e_steps > 0:
        src_pin = torch.from_numpy(s.view("int32")).pin_memory()
        dst_pin = torch.from_numpy(d.view("int32")).pin_memory()
    learned_line = None
    model = None
    if not args.no_learned and rank == 0:
        from paper_1209_6308_gb300 import learned
        log("training the cost model")
        model, minfo = learned.train_cost_model(scales=(18, 19, 20, 21, 22), steps=800, stream=sh)
        log(f"cost model trained: {minfo}")
        learned_line = learned_comparison(tc, g, stream, model, minfo)
        log("learned comparison done")
    e2e_ms = []
    e2e_counts = None
    log("end-to-end steps")
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = tc.tc_graph_create_arcs(n, src_pin, dst_pin, stream=sh, options=opts)
        c = tc.tc_census(h, stream=sh, options=opts_run)
        tc.tc_graph_destroy(h)
        dt = (time.perf_counter() - t0) * 1e3
        if i:
            e2e_ms.append(dt)
        e2e_counts = c
    g.close()
    e2e_job_ms = max_over_ranks(dist, statistics.mean(e2e_ms), "cuda") if e2e_ms else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    interval_line = None
    if not args.no_interval:
        log("interval census")
        interval_line = interval_comparison(tc, torch, s, d, n, sh)
    census64_line = None
    if not args.no_census64:
        log("64-state census")
        census64_line = census64_comparison(tc, torch, sh)
    serve_line = None
    if not args.no_serve:
        log("serving")
        serve_line = serving_comparison(tc, torch, sh, model, args)
        log("serving done")
    if model is not None:
        tc.tc_costmodel_destroy(model)

    peak, peak_kind = measured_peak()
    bytes_alg = info["bytes_alg"]
    achieved = bytes_alg / (ms * 1e-3) / 1e9
    traffic = stored_traffic()
    line = {
        "metric": METRIC, "value": job_value(world, arcs, ms),
        "unit": "arcs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "n": n, "arcs": arcs, "e_sym": info["e_sym"],
                   "algo": args.algo, "schedule": "plain", "l2": "flushed between steps (512 MB write)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "k_census", "bytes_alg_per_launch": bytes_alg},
        "e2e": ({"value": job_value(world, arcs, e2e_job_ms), "unit": "arcs/s",
                 "h2d_bytes_per_step": 8 * arcs, "d2h_bytes_per_step": 16 * 16,
                 "ms_per_step": e2e_job_ms} if e2e_ms else None),
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "census": counts,
        "census_e2e_equal": (e2e_counts == counts) if e2e_counts else None,
        "step_ms": {"min": min(step_ms), "max": max(step_ms)},
        "timed_wall_s": wall,
    }
    if learned_line is not None:
        line["learned"] = learned_line
    if interval_line is not None:
        line["interval"] = interval_line
    if census64_line is not None:
        line["census64"] = census64_line
    if serve_line is not None:
        line["serving"] = serve_line
    if not args.no_batch:
        log("batched comparison")
        line["batched"] = batched_comparison(tc, torch, sh, stream, args.autotune_trials)
    if not args.no_cpu_baseline:
        log("cpu baseline")
        line["cpu_baseline"] = cpu_baseline(n, s, d, arcs, args.cpu_sample_stride or CPU_STRIDE)
    log("done")
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

"""Benchmark of the GB300 triad census (one JSON line on rank 0).

A step is one full census (Fig. 5) of the R-MAT scale-26 workload, the largest single-GPU
configuration: n = 2^26, edge factor 16, a/b/c/d = .57/.19/.19/.05, ids permuted, loops and
duplicates dropped, 20% of arcs reciprocated, seed 3.  `value` is arcs/s with the CSR resident in
HBM (device time per census from CUDA events on the launching stream; the inputs are far larger
than L2 and a 512 MB write also flushes it between steps, outside the events) with the plain
schedule; the learned schedule is timed beside it (`learned`).  `e2e` is the same metric through
the public C ABI from pinned host arc buffers: graph build (H2D copy, symmetrise, dedupe,
relabel, sort) plus census plus the D2H read of the 16 counts, every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--scale 26|20|10] [--impl reference]

Under torchrun (N > 1) the census is sharded (paper Sec. 6-7: the connected pairs are
independent): every rank builds the same graph, runs its contiguous share of the work
(tc_census_shard) and the ranks sum their 16 counters with one NCCL all-reduce inside the timed
step; `value` is the graph's arcs over the slowest rank's step time (strong scaling).

--impl reference times the CPU oracle (test infrastructure; its OpenMP form on the host's cores)
on bounded samples of the same workload.
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
# R-MAT workloads by scale (edge factor 16, a/b/c = .57/.19/.19, ids permuted): scale 26 (the
# largest single-GPU configuration, plain vs learned) is the bench's default; scale 20 the medium
# configuration, reported as a section; scale 10 the small parity case
WORKLOADS = {10: dict(name="rmat10_ef16_r15_seed1", scale=10, edge_factor=16, recip=0.15, seed=1),
             20: dict(name="rmat20_ef16_r20_seed2", scale=20, edge_factor=16, recip=0.2, seed=2),
             26: dict(name="rmat26_ef16_r20_seed3", scale=26, edge_factor=16, recip=0.2, seed=3)}
WORKLOAD = dict(WORKLOADS[26])


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--algo", default="triangle", choices=["triangle", "suffix", "union"])
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--learned-reps", type=int, default=3, help="censuses per arm of the learned-vs-plain timing")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-seconds", type=float, default=12.0, help="target wall seconds of the CPU sample")
    p.add_argument("--no-batch", action="store_true", help="skip the 4096-graph batched comparison")
    p.add_argument("--autotune-trials", type=int, default=0, help="0 = the autotuner's whole search")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-schedule comparison")
    p.add_argument("--no-medium", action="store_true", help="skip the scale-20 section")
    p.add_argument("--no-forms", action="store_true", help="skip the suffix-form timing beside the headline form")
    p.add_argument("--no-serve", action="store_true", help="skip the serving (continuous batching) run")
    p.add_argument("--no-interval", action="store_true", help="skip the interval (windowed stream) census run")
    p.add_argument("--no-census64", action="store_true", help="skip the 64-state census run")
    p.add_argument("--no-matrix", action="store_true", help="skip the matrix-form census run")
    p.add_argument("--serve-seconds", type=float, default=60.0, help="measured seconds per serving arm")
    p.add_argument("--serve-warmup", type=float, default=5.0, help="unmeasured seconds before them")
    p.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate (requests/s)")
    p.add_argument("--serve-sweep", default="4000,8000,16000",
                   help="further arrival rates for a short plain-schedule sweep ('' = none)")
    p.add_argument("--sweep-seconds", type=float, default=8.0, help="measured seconds per sweep rate")
    p.add_argument("--scale", type=int, default=26, choices=sorted(WORKLOADS), help="R-MAT workload scale")
    a = p.parse_args(argv)
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
    """The slowest rank's time: the job's time when every rank works on its own share."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(arcs: int, ms: float) -> float:
    """Whole-job arcs/s of a sharded census: the graph's arcs over the slowest rank's time (every
    rank holds a share of one census, so the arcs are counted once)."""
    return arcs / (ms * 1e-3)


def bytes_alg_8d(n: int, info: dict) -> int:
    """Algorithmic bytes of one census by the scope contract's count: the CSR read once
    (8(n+1) offsets, 4 B per entry of the 2 e_sym list entries), each v list streamed per
    upper pair (4 d_v) plus 16 B of offsets and pair record, and the 16 counters."""
    return 8 * (n + 1) + 8 * info["e_sym"] + 4 * info["sum_dv_upper"] + 16 * info["e_sym"] + 128


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
def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the record of the CPU baseline."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def calibrate_stride(og, n: int, target_s: float, threads: int = 0) -> int:
    """A vertex stride whose OpenMP sample of the Fig. 5 loop lasts about target_s: start with a
    few dozen vertices and widen 8x at a time until a sample lasts target_s / 8, then scale."""
    stride = 1 << max(0, n.bit_length() - 6)
    while True:
        sec = og.sample_parallel(stride, 0, threads)[0]
        if sec >= target_s / 8 or stride == 1:
            break
        stride = max(1, stride // 8)
    return max(1, int(stride * min(1.0, max(sec, 1e-3) / target_s)))


def cpu_baseline(n, s, d, arcs, target_s):
    """The oracle's OpenMP form of Fig. 5 on every host core, on a vertex sample of the same
    graph (u = 0 mod stride, sized to about target_s of wall time), scaled to the full census by
    the sample's share of the merge work."""
    import oracle
    t0 = time.perf_counter()
    og = oracle.SampledGraph(n, s, d)
    build_s = time.perf_counter() - t0
    stride = calibrate_stride(og, n, target_s)
    sec, _, ws, wt, used = og.sample_parallel(stride, 0)
    og.close()
    frac = ws / wt if wt else 1.0
    full = sec / frac if frac > 0 else float("inf")
    return {"value": arcs / full, "unit": "arcs/s", "cores": used, "kind": "oracle",
            "cpu": cpu_model(), "nproc": os.cpu_count(),
            "sample": (f"the oracle's OpenMP form of Fig. 5 (dynamic schedule, private census vectors) on {used} "
                       f"threads over the vertices u = 0 (mod {stride}) of the same graph: {sec:.1f} s wall for "
                       f"{frac * 100:.4f}% of the union-walk work, scaled to the full census "
                       f"(oracle graph build {build_s:.0f} s, untimed)"),
            "full_census_estimate_s": full}


def run_reference(args):
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n, s, d = workload()
    arcs = len(s)
    og = oracle.SampledGraph(n, s, d)
    # stride for a few seconds of wall time per step, chosen before the steps
    stride = calibrate_stride(og, n, 3.0)
    secs, fracs, used = [], [], 1
    for i in range(args.warmup + args.steps):
        sec, _, ws, wt, used = og.sample_parallel(stride, i % stride)
        if i >= args.warmup:
            secs.append(sec)
            fracs.append(ws / wt if wt else 1.0)
    og.close()
    t = sum(secs) / sum(fracs)         # pooled estimate of the full-census time
    v = arcs / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "arcs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "n": n, "arcs": arcs},
            "cpu_baseline": {"value": v, "unit": "arcs/s", "cores": used, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"step i: the oracle's OpenMP form of Fig. 5 on {used} threads over u = i "
                                       f"(mod {stride}); full-census time estimated as total sample seconds / "
                                       f"total work fraction ({sum(fracs) * 100:.4f}% of the union-walk work)"},
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


KERNEL_SRC = {"k_census": "census.cu", "k_triangles": "triangles.cu"}


def traffic_file(workload_name: str, kernel: str = "k_census") -> str:
    return os.path.join(ROOT, "profiles", f"{kernel}_{workload_name.split('_')[0]}_traffic.txt")


def stored_traffic(workload_name: str = "rmat20_ef16_r20_seed2", kernel: str = "k_census"):
    """Per-launch DRAM bytes of a kernel on a workload from the committed ncu summary, if it was
    taken on the current code of the kernel's source file (else None)."""
    try:
        src = os.path.join(ROOT, "paper_1209_6308_gb300", "csrc", KERNEL_SRC[kernel])
        kv = dict(line.split(":", 1) for line in open(traffic_file(workload_name, kernel)) if ":" in line)
        if kv.get("code_sha256_16", kv.get("census_code_sha256_16", "")).strip() == census_code_hash(open(src).read()):
            return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def batched_comparison(tc, torch, sh, st, trials):
    """4096 Chung-Lu graphs (n log-uniform in [32, 65536], exponent 2.1, mean degree 8, 10%
    reciprocated, seed 4): a per-graph launch loop vs one persistent graph-captured launch over
    all of them, each in the suffix and the triangle form, and the autotuned launch (started
    from the triangle form).  All must give identical counts."""
    import graphgen
    specs = graphgen.batch_chung_lu(4096, 32, 65536, 8.0, 2.1, 0.1, 4)
    arcs = int(sum(len(s) for (_, s, _) in specs))
    gs = [tc.Graph.from_arcs(n, s, d, stream=sh, options={"algo": tc.TC_ALGO_TRIANGLE}) for (n, s, d) in specs]
    handles = [g.handle for g in gs]
    k = len(gs)
    ref_out = torch.zeros(16 * k, dtype=torch.int64, device="cuda")
    out = torch.zeros(16 * k, dtype=torch.int64, device="cuda")

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

    stats = [g.stats() for g in gs]
    res = {"workload": "chunglu4096_n32-65536_g2.1_d8_r10_seed4", "graphs": k, "arcs": arcs}
    same = True
    for name, algo in (("suffix", tc.TC_ALGO_SUFFIX), ("triangle", tc.TC_ALGO_TRIANGLE)):
        o = {"algo": algo}
        dst = ref_out if name == "suffix" else out

        def loop():
            for i, h in enumerate(handles):
                tc.tc_census_async(h, dst[16 * i:16 * i + 16], stream=sh, options=o)

        loop_ms = timed(loop, 2)
        same &= name == "suffix" or bool(torch.equal(out, ref_out))
        b = tc.tc_batch_create(handles, stream=sh, options=o)
        try:
            batch_ms = timed(lambda: tc.tc_batch_census_async(b, out, stream=sh), 5)
            same &= bool(torch.equal(out, ref_out))
            n_items, n_blocks = tc.tc_batch_stats(b)
        finally:
            tc.tc_batch_destroy(b)
        own = sum(st["bytes_alg_tri" if algo == tc.TC_ALGO_TRIANGLE else "bytes_alg"] for st in stats)
        res[name] = {"per_graph_loop": {"ms": loop_ms, "arcs_per_s": arcs / (loop_ms * 1e-3), "launches": k},
                     "persistent": {"ms": batch_ms, "arcs_per_s": arcs / (batch_ms * 1e-3), "launches": 1,
                                    "items": n_items, "warp_blocks": n_blocks},
                     "speedup_vs_loop": loop_ms / batch_ms,
                     "roofline": roofline_hbm(own, batch_ms, f"batched launch, {name} form", None, "issue")}
    b = tc.tc_batch_create(handles, stream=sh, options={"algo": tc.TC_ALGO_TRIANGLE})
    try:
        t0 = time.perf_counter()
        best, _ = tc.tc_batch_autotune(b, max_trials=trials, stream=sh)
        tune_s = time.perf_counter() - t0
        hist = tc.tc_batch_autotune_history(b)
        tuned_ms = timed(lambda: tc.tc_batch_census_async(b, out, stream=sh), 5)
        same &= bool(torch.equal(out, ref_out))
    finally:
        tc.tc_batch_destroy(b)
        for g in gs:
            g.close()
    res["persistent_autotuned"] = {"ms": tuned_ms, "arcs_per_s": arcs / (tuned_ms * 1e-3), "best": best,
                                   "tuning_s": tune_s, "trials": len(hist),
                                   "default_ms": hist[0][1] if hist else None,
                                   "trial_ms": [[o["algo"], o["warp_max_deg"], o["chunk_entries"], o["ctas_per_sm"],
                                                 o["item_work"], round(ms, 3)] for o, ms in hist]}
    res["speedup_vs_loop"] = res["suffix"]["per_graph_loop"]["ms"] / min(res["triangle"]["persistent"]["ms"], tuned_ms)
    res["counts_identical"] = same
    return res


def learned_comparison(tc, g, stream, model, info, reps, algo):
    """Cost model trained on R-MAT scales 18-22 (seeds 18-22) from cycles the plain census of the
    same kernel form measures, attached to the bench graph: census time with the plain and the
    learned schedule (identical counts required), each arm's roofline, and the held-out
    cost-prediction error."""
    from paper_1209_6308_gb300 import learned
    plain, learn = {"algo": algo}, {"algo": algo, "schedule": tc.TC_SCHED_LEARNED}
    learned.attach(model, g, stream=stream.cuda_stream)
    plain_ms, plain_c = learned.census_ms(g, plain, stream, reps=reps)
    learned_ms, learned_c = learned.census_ms(g, learn, stream, reps=reps)
    q = learned.prediction_quality(model, g, options=plain, stream=stream.cuda_stream)
    bal_plain = learned.balance(g, plain, stream=stream.cuda_stream)
    bal_learned = learned.balance(g, learn, stream=stream.cuda_stream)
    return {"_plain_counts": plain_c, "training": info, "plain_ms": plain_ms, "learned_ms": learned_ms, "reps": reps,
            "speedup": plain_ms / learned_ms, "counts_identical": plain_c == learned_c,
            "balance_plain": bal_plain, "balance_learned": bal_learned,
            "plain_arcs_per_s": None, "learned_arcs_per_s": None,
            "roofline_plain": form_roofline(tc, g.n, g.stats(), algo, plain_ms),
            "roofline_learned": form_roofline(tc, g.n, g.stats(), algo, learned_ms),
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


def serving_comparison(tc, torch, sh, model, args, algo):
    """Serving workload with the plain and the learned schedule (the bench's kernel form):
    p50/p99 latency and arcs/s, and a short sweep of higher arrival rates."""
    from paper_1209_6308_gb300 import learned
    t0 = time.perf_counter()
    pool = serving_pool()
    gen_s = time.perf_counter() - t0
    log(f"serving pool generated in {gen_s:.1f}s")
    plain = {"algo": algo}
    learn = {"algo": algo, "schedule": tc.TC_SCHED_LEARNED}
    gs = [tc.Graph.from_arcs(n, s, d, stream=sh, options=plain) for (_, (n, s, d)) in pool]
    arcs = [len(s) for (_, (_, s, _)) in pool]
    want = [g.census(stream=sh, options=plain) for g in gs]
    out = {"workload": SERVE_POOL + f"_poisson{int(args.serve_rate)}_seed5", "graphs": len(gs),
           "pool_arcs": int(sum(arcs)), "rate_per_s": args.serve_rate, "measured_s": args.serve_seconds,
           "warmup_s": args.serve_warmup, "quantum_us": 1000, "lanes": 3, "pool_generation_s": gen_s,
           "selection": "graph i with probability proportional to 1/arcs_i", "kernel_form": FORM_NAMES[algo]}
    try:
        arms = [("plain", plain)]
        if model is not None:
            for g in gs:
                learned.attach(model, g, stream=sh)
            arms.append(("learned", learn))
        exact = True
        for name, opts in arms:
            log(f"serving arm {name}")
            m, res, rid_graph = serve_arm(tc, gs, arcs, opts, args.serve_rate, args.serve_seconds,
                                          args.serve_warmup, 5)
            exact &= all(r.census() == want[rid_graph[r.id][1]] for r in res)
            out[name] = m
        # the plain schedule at higher arrival rates, briefly: where does the p99 pass 10 ms?
        sweep = []
        rates = [float(x) for x in args.serve_sweep.split(",") if x.strip()]
        for rate in rates:
            log(f"serving sweep at {rate:.0f} req/s")
            m, res, rid_graph = serve_arm(tc, gs, arcs, plain, rate, args.sweep_seconds, 2.0, 6)
            exact &= all(r.census() == want[rid_graph[r.id][1]] for r in res)
            sweep.append({"rate_per_s": rate, "measured_s": args.sweep_seconds, "warmup_s": 2.0,
                          **{k: m.get(k) for k in ("requests", "p50_ms", "p99_ms", "max_ms", "arcs_per_s",
                                                   "offered_arcs_per_s", "achieved_rate", "gpu_busy_frac",
                                                   "overloaded")}})
        if sweep:
            out["sweep_plain"] = sweep
            pts = [(out["rate_per_s"], out["plain"].get("p99_ms"))] + [(x["rate_per_s"], x["p99_ms"]) for x in sweep]
            over = [r for r, p99 in pts if p99 is None or p99 > 10.0]
            out["p99_above_10ms_first_rate"] = min(over) if over else None
        out["counts_identical_to_standalone"] = exact
    finally:
        for g in gs:
            g.close()
    return out


def interval_comparison(tc, torch, s, d, n, sh, name, window=200, every=10):
    """Interval census (the paper's monitoring use): the bench graph's arcs in a random order at
    uniform times over [0, 1000), a window of 200, a census every 10 from 200 to 1000.  Each
    census merges the arcs that entered and left since the last one into the window's kept arc
    set, builds the window's graph from it and counts it (about a fifth of the arcs per window,
    a twentieth of those changed per step).  Beside it, every tenth window rebuilt from its arcs
    with tc_graph_create_arcs (device arrays) and counted, as a census without the kept set
    would; both must give the same counts."""
    import numpy as np
    rng = np.random.default_rng(7)
    perm = rng.permutation(len(s))
    t = np.sort(rng.integers(0, 1000, len(s))).astype(np.uint64)
    src, dst = s[perm], d[perm]
    opts = {"algo": tc.TC_ALGO_TRIANGLE}
    times, windows, got = [], [], {}
    with tc.Stream(n, window, options=opts, stream=sh) as st:
        t0 = time.perf_counter()
        st.push(src, dst, t)
        push_s = time.perf_counter() - t0
        for t_now in range(window, 1001, every):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            c, m = st.census(t_now)
            times.append((time.perf_counter() - t1) * 1e3)
            windows.append(m)
            got[t_now] = c
        info = st.stats()
    sd = torch.from_numpy(src.view("int32")).cuda()
    dd = torch.from_numpy(dst.view("int32")).cuda()
    full_times, same = [], True
    for t_now in range(window, 1001, 10 * every):
        a = int(np.searchsorted(t, t_now - window, side="right"))
        b = int(np.searchsorted(t, t_now, side="right"))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h = tc.tc_graph_create_arcs(n, sd[a:b], dd[a:b], stream=sh, options=opts)
        c = tc.tc_census(h, stream=sh, options=opts)
        full_times.append((time.perf_counter() - t1) * 1e3)
        tc.tc_graph_destroy(h)
        same = same and c == got[t_now]
    del sd, dd
    ms = statistics.median(times[1:])
    full_ms = statistics.median(full_times)
    return {"workload": f"{name}_times_uniform1000_window{window}_every{every}", "censuses": len(times),
            "arcs_per_window_median": int(statistics.median(windows)), "ms_per_census_median": ms,
            "first_census_ms": times[0], "arcs_per_s": statistics.median(windows) / (ms * 1e-3), "push_s": push_s,
            "set_rebuilds": info["rebuilds"], "set_repairs": info["repairs"],
            "arcs_changed_last_census": info["last_added"] + info["last_evicted"],
            "rebuild_from_arcs_ms_median": full_ms, "speedup_vs_rebuild": full_ms / ms,
            "counts_identical_to_rebuild": same,
            "note": "per census: merge of the entering and leaving arcs into the kept arc set, the window's "
                    "graph from it (pairs, degrees, relabel, CSR, tables), census, D2H of 16 counts; "
                    "wall time of the synchronous call"}


def census64_comparison(tc, torch, sh, scale, steps=3):
    """The 64-state census (Sec. 3, Fig. 2) of an R-MAT graph (ef16, 20% recip, seed = scale).
    Timed with CUDA events around the synchronous call (id inversion, census, 1 KB D2H);
    checked by folding the 64 states into the 16 classes and comparing with the census of the
    same graph."""
    import graphgen
    n, s, d = graphgen.rmat(scale, 16, 0.2, scale)
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
    return {"workload": f"rmat{scale}_ef16_r20_seed{scale}", "n": n, "arcs": len(s), "ms": ms,
            "arcs_per_s": len(s) / (ms * 1e-3), "fold_equals_census16": fold == c16,
            "roofline": dict(roofline_hbm(bytes_alg_8d(n, info), ms, "census64 (sort, wedges, triangle walk)", None,
                                          "issue"),
                             note="bytes: the scope formula of the 16-class census (each pair streams its v list)")}


def matrix_comparison(tc, torch, sh, steps=3):
    """The matrix form of the census (Sec. 4, tc_census_matrix) on R-MAT scale 14 (ef16, 20%
    recip, seed 14; n = 2^14, the largest it takes): time per call (CUDA events around the
    synchronous call: bit matrices, six masked products, 24 sums to the host) and agreement with
    the triangle form of the Fig. 5 census on the same graph."""
    import graphgen
    n, s, d = graphgen.rmat(14, 16, 0.2, 14)
    from paper_1209_6308_gb300 import learned
    st = torch.cuda.ExternalStream(sh)
    with tc.Graph.from_arcs(n, s, d, stream=sh, options={"algo": tc.TC_ALGO_TRIANGLE}) as g:
        c16 = g.census(stream=sh)
        cm = g.census_matrix(stream=sh)
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            cm = g.census_matrix(stream=sh)
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        tri_ms, _ = learned.census_ms(g, {"algo": tc.TC_ALGO_TRIANGLE}, torch.cuda.Stream(), reps=5)
    ms = statistics.median(times)
    W = (n + 63) // 64
    words = 6 * n * n * W       # AND + popcount word operations of the six products
    return {"workload": "rmat14_ef16_r20_seed14", "n": n, "arcs": len(s), "ms": ms, "equals_census16": cm == c16,
            "triangle_form_ms": tri_ms, "and_popc_words_per_s": words / (ms * 1e-3)}


def roofline_hbm(bytes_alg: int, ms: float, kernel: str, traffic=None, bound="hbm") -> dict:
    peak, peak_kind = measured_peak()
    achieved = bytes_alg / (ms * 1e-3) / 1e9
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel, "bytes_alg_per_launch": bytes_alg}


FORM_NAMES = {0: "union", 1: "suffix", 2: "triangle"}


def form_roofline(tc, n, info, algo, ms):
    """Roofline of one census.  `bytes_alg_per_launch` is what the kernel form itself must read
    (tc_graph_info: the triangle form's or the suffix form's count; the scope contract's count
    for the union walk, which reads what it describes), so `frac` compares the form with
    streaming its own data at copy speed.  The scope contract's count (every pair streams its
    v list, the paper's walk) is given beside it as `contract_*`: a form that skips most of
    that reading can exceed 1 there."""
    kernel = {tc.TC_ALGO_TRIANGLE: "k_triangles", tc.TC_ALGO_SUFFIX: "k_census (suffix)"}.get(algo, "k_census (union)")
    b8d = bytes_alg_8d(n, info)
    own = {tc.TC_ALGO_TRIANGLE: info["bytes_alg_tri"], tc.TC_ALGO_SUFFIX: info["bytes_alg"]}.get(algo, b8d)
    r = roofline_hbm(own, ms, kernel, None, "issue")
    r["contract_bytes_per_launch"] = b8d
    r["contract_achieved"] = b8d / (ms * 1e-3) / 1e9
    r["contract_frac"] = r["contract_achieved"] / r["peak"]
    return r


def medium_section(tc, torch, stream, steps=5):
    """The scale-20 workload (configuration 2): census time of each kernel form (plain
    schedule), with rooflines; all three must give the same counts."""
    import graphgen
    sh = stream.cuda_stream
    n, s, d = graphgen.rmat(20, 16, 0.2, 2)
    from paper_1209_6308_gb300 import learned
    out = {"workload": WORKLOADS[20]["name"], "n": n, "arcs": len(s)}
    counts = {}
    with tc.Graph.from_arcs(n, s, d, stream=sh) as g:        # created without options: the union walk by default
        info = g.stats()
        out["e_sym"] = info["e_sym"]
        for algo in (tc.TC_ALGO_TRIANGLE, tc.TC_ALGO_SUFFIX, tc.TC_ALGO_UNION):
            ms, c = learned.census_ms(g, {"algo": algo} if algo else None, stream, reps=steps if algo else 3)
            counts[algo] = c
            out[FORM_NAMES[algo]] = {"ms": ms, "arcs_per_s": len(s) / (ms * 1e-3),
                                     "roofline": form_roofline(tc, n, info, algo, ms)}
    c = counts[tc.TC_ALGO_TRIANGLE]
    out["forms_agree"] = all(v == c for v in counts.values())
    c[0] = tc.tc_null_count(n, c)
    out["census"] = c
    return out


def run_gpu(args):
    import torch
    import paper_1209_6308_gb300 as tc
    from paper_1209_6308_gb300 import shard

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    algo = {"triangle": tc.TC_ALGO_TRIANGLE, "suffix": tc.TC_ALGO_SUFFIX, "union": tc.TC_ALGO_UNION}[args.algo]
    opts = {"algo": algo}
    log("generating the workload")
    t0 = time.perf_counter()
    n, s, d = workload()
    gen_s = time.perf_counter() - t0
    arcs = len(s)
    log(f"workload: n={n} arcs={arcs} ({gen_s:.1f}s)")
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    t0 = time.perf_counter()
    g = tc.Graph.from_arcs(n, s, d, stream=sh, options=opts)
    build_s = time.perf_counter() - t0
    info = g.stats()
    log(f"graph built in {build_s:.1f}s: e_sym={info['e_sym']} sum_walk={info['sum_walk']}")
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def one_step():
        # this rank's shard of the census (the whole census at world 1), then the sum of the
        # ranks' 16 counters: the one collective of the path
        if world == 1:
            tc.tc_census_async(g.handle, out, stream=sh, options=opts)
        else:
            shard.enqueue_shard(g, out, rank, world, stream=sh, options=opts)
            shard.allreduce_counts(dist, out)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            one_step()
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
                one_step()
                ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = max_over_ranks(dist, statistics.mean(step_ms), "cuda")
    counts = shard.census_of_sum(n, out.cpu())
    log(f"timed: {ms:.2f} ms per step")

    # end to end through the C ABI from pinned host buffers
    e2e_ms, e2e_build_ms, e2e_counts = [], [], None
    if args.e2e_steps > 0:
        src_pin = torch.from_numpy(s.view("int32")).pin_memory()
        dst_pin = torch.from_numpy(d.view("int32")).pin_memory()
        log("end-to-end steps")
        for i in range(args.e2e_steps + 1):
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = tc.tc_graph_create_arcs(n, src_pin, dst_pin, stream=sh, options=opts)
            t_built = time.perf_counter()
            if world == 1:
                c = tc.tc_census(h, stream=sh, options=opts)
            else:
                with torch.cuda.stream(stream):
                    c = shard.sharded_census(h, n, out, rank, world, dist, stream=stream, options=opts)
            dt = (time.perf_counter() - t0) * 1e3
            tc.tc_graph_destroy(h)
            if i:
                e2e_ms.append(dt)
                e2e_build_ms.append((t_built - t0) * 1e3)
            e2e_counts = c
        del src_pin, dst_pin
    e2e_job_ms = max_over_ranks(dist, statistics.mean(e2e_ms), "cuda") if e2e_ms else None

    if rank != 0:
        g.close()
        if dist:
            dist.destroy_process_group()
        return 0

    learned_line, model = None, None
    if not args.no_learned:
        from paper_1209_6308_gb300 import learned
        log("training the cost model")
        model, minfo = learned.train_cost_model(scales=(18, 19, 20, 21, 22), steps=800, stream=sh, options=opts)
        log(f"cost model trained: {minfo}")
        learned_line = learned_comparison(tc, g, stream, model, minfo, args.learned_reps, algo)
        learned_line["kernel_form"] = args.algo
        learned_line["plain_arcs_per_s"] = arcs / (learned_line["plain_ms"] * 1e-3)
        learned_line["learned_arcs_per_s"] = arcs / (learned_line["learned_ms"] * 1e-3)
        learned_line["counts_identical_to_timed"] = learned_line.pop("_plain_counts")[1:] == counts[1:]
        log("learned comparison done")
    forms_line = None
    if not args.no_forms and algo != tc.TC_ALGO_SUFFIX:
        from paper_1209_6308_gb300 import learned
        log("suffix form timing")
        ms_suf, c_suf = learned.census_ms(g, {"algo": tc.TC_ALGO_SUFFIX}, stream, reps=2)
        forms_line = {"suffix": {"ms": ms_suf, "arcs_per_s": arcs / (ms_suf * 1e-3),
                                 "roofline": form_roofline(tc, n, info, tc.TC_ALGO_SUFFIX, ms_suf),
                                 "counts_equal": c_suf[1:] == counts[1:]},
                      FORM_NAMES[algo]: {"ms": ms, "arcs_per_s": arcs / (ms * 1e-3)},
                      "speedup": ms_suf / ms}
    g.close()
    del flush
    torch.cuda.empty_cache()

    medium_line = None
    if not args.no_medium and WORKLOAD["scale"] != 20:
        log("scale-20 section")
        medium_line = medium_section(tc, torch, stream)
    interval_line = None
    if not args.no_interval:
        log("interval census")
        import graphgen
        wl = WORKLOAD if WORKLOAD["scale"] <= 20 else WORKLOADS[20]
        ni, si, di = (n, s, d) if WORKLOAD["scale"] <= 20 else graphgen.rmat(20, 16, 0.2, 2)
        interval_line = interval_comparison(tc, torch, si, di, ni, sh, wl["name"])
    matrix_line = None
    if not args.no_matrix:
        log("matrix census")
        matrix_line = matrix_comparison(tc, torch, sh)
    census64_lines = None
    if not args.no_census64:
        census64_lines = []
        for sc in (16, 20):
            log(f"64-state census, scale {sc}")
            census64_lines.append(census64_comparison(tc, torch, sh, sc))
    serve_line = None
    if not args.no_serve:
        log("serving")
        serve_line = serving_comparison(tc, torch, sh, model, args, algo)
        log("serving done")
    if model is not None:
        tc.tc_costmodel_destroy(model)

    kernel = "k_triangles" if algo == tc.TC_ALGO_TRIANGLE else "k_census"
    traffic = stored_traffic(WORKLOAD["name"], kernel)
    roof = form_roofline(tc, n, info, algo, ms)
    roof["traffic"] = traffic
    roof["note"] = ("bytes_alg_per_launch = what this kernel form reads (tc_graph_info bytes_alg_tri: "
                    "32(n+1) + 60 E + 4 sum_tri_walk + 1280); contract_* = the scope formula 8(n+1) + 8 E + "
                    "sum over upper pairs (4 d_v + 16) + 128 (each pair streams N[v], the paper's walk), which "
                    "this form does not read; the kernel is bound by load latency and instruction issue (ncu), "
                    "not by HBM bandwidth")
    line = {
        "metric": METRIC, "value": job_value(arcs, ms),
        "unit": "arcs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "n": n, "arcs": arcs, "e_sym": info["e_sym"],
                   "algo": args.algo, "schedule": "plain",
                   "l2": "inputs far larger than L2 (CSR and tables); also flushed between steps (512 MB write)",
                   "parallelism": f"shard{world}" if world > 1 else "single"},
        "roofline": roof,
        "e2e": ({"value": job_value(arcs, e2e_job_ms), "unit": "arcs/s",
                 "h2d_bytes_per_step": 8 * arcs, "d2h_bytes_per_step": 16 * 16,
                 "ms_per_step": e2e_job_ms,
                 "build_ms": statistics.mean(e2e_build_ms) if e2e_build_ms else None,
                 "path": "tc_graph_create_arcs from page-locked host arcs (read by the build's key kernel over "
                         "the host link), tc_census (plan + census), 16 counts to the host"} if e2e_ms else None),
        # per census: k_pair_bulk, k_triangles, k_tri_fold (triangle form) or k_census
        "gpu_launches": args.steps * (3 if algo == tc.TC_ALGO_TRIANGLE else 1),
        "clocks": clk.summary(),
        "census": counts,
        "census_e2e_equal": (e2e_counts == counts) if e2e_counts else None,
        "step_ms": {"min": min(step_ms), "max": max(step_ms)},
        "timed_wall_s": wall, "generate_s": gen_s, "build_s": build_s,
    }
    if learned_line is not None:
        line["learned"] = learned_line
    if forms_line is not None:
        line["forms"] = forms_line
    if medium_line is not None:
        line["medium"] = medium_line
    if interval_line is not None:
        line["interval"] = interval_line
    if census64_lines is not None:
        line["census64"] = census64_lines
    if matrix_line is not None:
        line["matrix"] = matrix_line
    if serve_line is not None:
        line["serving"] = serve_line
    if not args.no_batch:
        log("batched comparison")
        line["batched"] = batched_comparison(tc, torch, sh, stream, args.autotune_trials)
    if not args.no_cpu_baseline:
        log("cpu baseline")
        line["cpu_baseline"] = cpu_baseline(n, s, d, arcs, args.cpu_sample_seconds)
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

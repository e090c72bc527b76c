"""Writes the stored census fixtures in this folder.  Calls only the CPU oracle and the
seeded generators; run from the repository root:

    python tests/golden/make_golden.py            # the small fixtures (seconds)
    python tests/golden/make_golden.py --s20      # scale-20 R-MAT workload (OpenMP oracle, ~20 min on 8 cores)
    python tests/golden/make_golden.py --batch    # the 4096 Chung-Lu graphs of the batched workload

The large fixtures use the oracle's OpenMP form of Fig. 5 (flattened loops, dynamic schedule,
private census vectors, Sec. 6-7), which the CPU tests pin bit-identical to the serial form;
the batch runs the serial form on several graphs at once (ctypes releases the GIL)."""
import argparse
import concurrent.futures as cf
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

S20_FILE = "rmat_s20_r20_seed2.txt"
BATCH_FILE = "chunglu_batch4096_seed4.txt"


def write(name, header, n, s, d, counts=None):
    c = counts if counts is not None else oracle.census_bm(n, s, d)
    with open(os.path.join(HERE, name), "w") as f:
        f.write(header)
        f.write(f"n {n}\narcs {len(s)}\n")
        for k, v in zip(oracle.CLASS_NAMES, c):
            f.write(f"{k} {v}\n")


def small():
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    write("rmat_s10_r15_seed1.txt",
          "# 16-type census (Fig. 5 method, Sec. 4) of the scale-10 R-MAT workload:\n"
          "# a/b/c/d = .57/.19/.19/.05, edge factor 16, ids permuted, loops and duplicates\n"
          "# dropped, 15% of arcs reciprocated, seed 1.  Written by make_golden.py from the\n"
          "# CPU oracle; cross-checked there against networkx.triadic_census.\n", n, s, d)
    n, s, d = graphgen.chung_lu(5000, 8.0, 2.1, 0.1, 4, 11)
    write("chunglu_n5000_seed4_g11.txt",
          "# 16-type census of a Chung-Lu digraph: n=5000, exponent 2.1, mean degree 8,\n"
          "# 10% reciprocated, seed 4, graph index 11.  Written by make_golden.py (oracle).\n", n, s, d)


def s20(threads):
    n, s, d = graphgen.rmat(20, 16, 0.2, 2)
    t0 = time.time()
    c = oracle.census_bm_parallel(n, s, d, threads)
    dt = time.time() - t0
    write(S20_FILE,
          "# 16-type census (Fig. 5 method, Sec. 4) of the scale-20 R-MAT workload:\n"
          "# n = 2^20, edge factor 16, a/b/c/d = .57/.19/.19/.05, ids permuted, loops and\n"
          "# duplicates dropped, 20% of arcs reciprocated, seed 2.  Written by make_golden.py\n"
          f"# with the CPU oracle's OpenMP form of Fig. 5 ({dt:.0f} s on {threads or os.cpu_count()} threads).\n",
          n, s, d, c)


def _one(spec):
    n, s, d = spec
    return oracle.census_bm(n, s, d)


def batch(threads):
    specs = graphgen.batch_chung_lu(4096, 32, 65536, 8.0, 2.1, 0.1, 4)
    t0 = time.time()
    # largest graphs first, so that the pool ends evenly
    order = sorted(range(len(specs)), key=lambda i: -len(specs[i][1]))
    res = [None] * len(specs)
    with cf.ThreadPoolExecutor(max_workers=threads or os.cpu_count()) as ex:
        for i, c in zip(order, ex.map(lambda i: _one(specs[i]), order)):
            res[i] = c
    dt = time.time() - t0
    with open(os.path.join(HERE, BATCH_FILE), "w") as f:
        f.write("# 16-type census (Fig. 5 method, Sec. 4) of each graph of the batched workload:\n"
                "# 4096 directed Chung-Lu graphs, n log-uniform in [32, 65536] (seed 4), exponent 2.1,\n"
                "# mean degree 8, 10% reciprocated, seed 4, graph index i.  Written by make_golden.py\n"
                f"# with the serial CPU oracle ({dt:.0f} s over {threads or os.cpu_count()} threads).\n"
                "# columns: i n arcs 003 012 102 021D 021U 021C 111D 111U 030T 030C 201 120D 120U 120C 210 300\n")
        for i, ((n, s, _), c) in enumerate(zip(specs, res)):
            f.write(f"{i} {n} {len(s)} " + " ".join(str(x) for x in c) + "\n")


def read_counts(name):
    """(n, arcs, 16 counts) of a single-graph fixture."""
    kv = {}
    for line in open(os.path.join(HERE, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        kv[k] = int(v)
    return kv["n"], kv["arcs"], [kv[c] for c in oracle.CLASS_NAMES]


def read_batch(name=BATCH_FILE):
    """List of (n, arcs, 16 counts), one per graph of the batched fixture."""
    out = []
    for line in open(os.path.join(HERE, name)):
        if line.startswith("#") or not line.strip():
            continue
        f = [int(x) for x in line.split()]
        assert f[0] == len(out)
        out.append((f[1], f[2], f[3:19]))
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--s20", action="store_true")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    if not (a.s20 or a.batch):
        small()
    if a.batch:
        batch(a.threads)
    if a.s20:
        s20(a.threads)

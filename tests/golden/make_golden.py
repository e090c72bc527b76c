"""Writes the stored census fixtures in this folder.  Calls only the CPU oracle and the
seeded generators; run from the repository root: python tests/golden/make_golden.py"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, header, n, s, d):
    c = oracle.census_bm(n, s, d)
    with open(os.path.join(HERE, name), "w") as f:
        f.write(header)
        f.write(f"n {n}\narcs {len(s)}\n")
        for k, v in zip(oracle.CLASS_NAMES, c):
            f.write(f"{k} {v}\n")


if __name__ == "__main__":
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

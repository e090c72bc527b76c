"""Pins for the CPU oracle (no GPU): it must agree with facts that do not come from itself.

Pins used: two independent tricode tables and their orbit sizes; the O(n^3) definition
(exhaustive on all 4096 digraphs with 4 vertices, random graphs up to n=64); closed forms
for graph families; weighted-sum identities against O(m) statistics; relabelling,
reversal and complement symmetries; networkx's independent triadic_census where
networkx is installed.
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from census_facts import (COMPLEMENT, ORBIT, REVERSE, check_invariants, choose2, choose3,
                          permute_classes)

T003, T012, T102, T021D, T021U, T021C, T111D, T111U, T030T, T030C, T201, T120D, T120U, T120C, T210, T300 = range(16)


def arcs_of(pairs):
    if not pairs:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    a = np.array(pairs, dtype=np.uint32)
    return a[:, 0].copy(), a[:, 1].copy()


def one_hot(n_total, k):
    v = [0] * 16
    v[k] = n_total
    return v


# ------------------------------------------------------------------ tables

def test_tables_agree_and_orbits():
    r, c = oracle.table_rules(), oracle.table_canonical()
    assert (r == c).all()
    assert list(np.bincount(r, minlength=16)) == ORBIT


def test_every_3_vertex_digraph_is_one_hot():
    """All 64 digraphs on 3 vertices: each census has exactly one triad, in its class."""
    T = oracle.table_rules()
    links = [(1, 0), (0, 1), (1, 2), (2, 1), (0, 2), (2, 0)]   # tricode bits 1..32 for (u,v,w)=(0,1,2)
    for code in range(64):
        pairs = [links[b] for b in range(6) if code >> b & 1]
        s, d = arcs_of(pairs)
        want = one_hot(1, int(T[code]))
        assert oracle.census_bm(3, s, d) == want, code
        assert oracle.census_brute(3, s, d) == want, code


def test_exhaustive_4_vertices_bm_equals_brute():
    ordered = [(a, b) for a in range(4) for b in range(4) if a != b]
    for mask in range(1 << 12):
        pairs = [ordered[i] for i in range(12) if mask >> i & 1]
        s, d = arcs_of(pairs)
        bm = oracle.census_bm(4, s, d)
        assert bm == oracle.census_brute(4, s, d), mask
        assert sum(bm) == 4


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [3, 5, 17, 100])
def test_empty_graph(n):
    s, d = arcs_of([])
    assert oracle.census_bm(n, s, d) == one_hot(choose3(n), T003)


@pytest.mark.parametrize("n", [3, 6, 40])
def test_complete_mutual(n):
    s, d = arcs_of([(a, b) for a in range(n) for b in range(n) if a != b])
    assert oracle.census_bm(n, s, d) == one_hot(choose3(n), T300)


@pytest.mark.parametrize("n", [3, 7, 50])
def test_transitive_tournament(n):
    s, d = arcs_of([(a, b) for a in range(n) for b in range(a + 1, n)])
    assert oracle.census_bm(n, s, d) == one_hot(choose3(n), T030T)


@pytest.mark.parametrize("n", [3, 8, 60])
def test_out_star_and_in_star(n):
    hub = n // 2
    s, d = arcs_of([(hub, x) for x in range(n) if x != hub])
    want = [0] * 16
    want[T021D] = choose2(n - 1)
    want[T003] = choose3(n - 1)
    assert oracle.census_bm(n, s, d) == want
    want_in = permute_classes(want, REVERSE)
    assert oracle.census_bm(n, d, s) == want_in
    assert want_in[T021U] == choose2(n - 1)


def test_directed_3_cycle():
    s, d = arcs_of([(0, 1), (1, 2), (2, 0)])
    assert oracle.census_bm(3, s, d) == one_hot(1, T030C)
    # embedded among 7 isolated vertices: each cycle arc meets 7 outsiders (012)
    c = oracle.census_bm(10, s, d)
    want = [0] * 16
    want[T030C], want[T012], want[T003] = 1, 21, choose3(10) - 22
    assert c == want


@pytest.mark.parametrize("n", [3, 4, 9, 64])
def test_directed_path(n):
    s, d = arcs_of([(i, i + 1) for i in range(n - 1)])
    c = oracle.census_bm(n, s, d)
    assert c[T021C] == n - 2
    assert c[T012] == (n - 1) * (n - 2) - 2 * (n - 2)
    assert c[T003] == choose3(n) - (n - 2) - c[T012]


def test_mutual_pair_plus_isolated():
    s, d = arcs_of([(0, 1), (1, 0)])
    c = oracle.census_bm(12, s, d)
    assert c[T102] == 10 and c[T003] == choose3(12) - 10


# ------------------------------------------------------------------ brute force on random graphs

@pytest.mark.parametrize("seed", range(8))
def test_random_gnp_matches_brute(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 65))
    p = float(rng.choice([0.02, 0.08, 0.25, 0.6]))
    n, s, d = graphgen.gnp(n, p, seed)
    assert oracle.census_bm(n, s, d) == oracle.census_brute(n, s, d)


@pytest.mark.parametrize("seed", range(1, 11))
def test_rmat_s10_induced_64_subgraphs_match_brute(seed):
    """The scale-10 workload's parity recipe: induced subgraphs on 64 random vertices."""
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    rng = np.random.default_rng(seed)
    keep = rng.choice(n, 64, replace=False)
    idx = -np.ones(n, np.int64)
    idx[keep] = np.arange(64)
    m = (idx[s] >= 0) & (idx[d] >= 0)
    ss, dd = idx[s[m]].astype(np.uint32), idx[d[m]].astype(np.uint32)
    assert oracle.census_bm(64, ss, dd) == oracle.census_brute(64, ss, dd)


def test_dirty_input_is_cleaned():
    """Loops and repeated arcs are ignored (the relation is a set)."""
    n, s, d = graphgen.gnp(30, 0.2, 5)
    s2 = np.concatenate([s, s[:50], np.arange(10, dtype=np.uint32)])
    d2 = np.concatenate([d, d[:50], np.arange(10, dtype=np.uint32)])
    perm = np.random.default_rng(0).permutation(len(s2))
    c, st = oracle.census_bm(n, s2[perm], d2[perm], with_stats=True)
    assert c == oracle.census_bm(n, s, d)
    assert st == (len(s), 10, 50)


def test_out_of_range_id_rejected():
    with pytest.raises(ValueError):
        oracle.census_bm(4, np.array([0, 4], np.uint32), np.array([1, 0], np.uint32))


# ------------------------------------------------------------------ invariants and symmetries

@pytest.mark.parametrize("make", ["rmat10", "chunglu", "gnp"])
def test_weighted_sum_invariants(make):
    if make == "rmat10":
        n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    elif make == "chunglu":
        n, s, d = graphgen.chung_lu(3000, 8.0, 2.1, 0.1, 4, 7)
    else:
        n, s, d = graphgen.gnp(200, 0.05, 9)
    check_invariants(n, oracle.census_bm(n, s, d), oracle.invariants(n, s, d))


def test_relabel_invariance():
    n, s, d = graphgen.rmat(9, 8, 0.2, 3)
    perm = np.random.default_rng(7).permutation(n).astype(np.uint32)
    assert oracle.census_bm(n, perm[s], perm[d]) == oracle.census_bm(n, s, d)


def test_reversal_swaps_up_and_down():
    n, s, d = graphgen.rmat(9, 8, 0.2, 4)
    assert oracle.census_bm(n, d, s) == permute_classes(oracle.census_bm(n, s, d), REVERSE)


@pytest.mark.parametrize("seed", range(3))
def test_complement_swaps_classes(seed):
    n, s, d = graphgen.gnp(40, 0.3, 20 + seed)
    adj = np.zeros((n, n), bool)
    adj[s, d] = True
    comp = ~adj
    np.fill_diagonal(comp, False)
    cs, cd = np.nonzero(comp)
    assert oracle.census_bm(n, cs.astype(np.uint32), cd.astype(np.uint32)) == \
        permute_classes(oracle.census_bm(n, s, d), COMPLEMENT)


def test_parallel_form_matches_serial():
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    assert oracle.census_bm_parallel(n, s, d, 4) == oracle.census_bm(n, s, d)


def test_sampled_timing_covers_the_whole_census_when_stride_is_one():
    n, s, d = graphgen.rmat(8, 16, 0.2, 2)
    sec, part, ws, wt = oracle.census_bm_sample(n, s, d, 1, 0)
    full = oracle.census_bm(n, s, d)
    assert ws == wt and part[1:] == full[1:] and sec >= 0


def test_samples_partition_the_census():
    """Samples over u = k (mod 5), k = 0..4, add up to the connected part of the census."""
    n, s, d = graphgen.rmat(9, 16, 0.2, 3)
    og = oracle.SampledGraph(n, s, d)
    tot, work = [0] * 16, 0
    for k in range(5):
        _, part, ws, wt = og.sample(5, k)
        tot = [a + b for a, b in zip(tot, part)]
        work += ws
    assert work == wt and tot[1:] == oracle.census_bm(n, s, d)[1:]


def test_parallel_samples_partition_the_census_like_the_serial_ones():
    """The OpenMP form of the timing sample (the paper's CPU form) gives the same partial
    counts and work as the serial sample, and its samples over u = k (mod 4) add up to the
    connected part of the census."""
    n, s, d = graphgen.rmat(9, 16, 0.2, 3)
    og = oracle.SampledGraph(n, s, d)
    tot, work = [0] * 16, 0
    for k in range(4):
        sec, part, ws, wt, used = og.sample_parallel(4, k, threads=3)
        _, part1, ws1, wt1 = og.sample(4, k)
        assert part == part1 and ws == ws1 and wt == wt1 and sec >= 0 and used >= 1
        tot = [a + b for a, b in zip(tot, part)]
        work += ws
    og.close()
    assert work == wt and tot[1:] == oracle.census_bm(n, s, d)[1:]


def test_unsorted_and_sorted_inputs_build_the_same_graph():
    """The oracle skips its sort for inputs already sorted by (src, dst): the census is the
    same for a shuffled copy with duplicates and loops."""
    n, s, d = graphgen.rmat(9, 16, 0.2, 3)
    rng = np.random.default_rng(1)
    s2 = np.concatenate([s, s[:50], np.arange(5, dtype=np.uint32)])
    d2 = np.concatenate([d, d[:50], np.arange(5, dtype=np.uint32)])
    p = rng.permutation(len(s2))
    a = oracle.census_bm(n, s, d, with_stats=True)
    b = oracle.census_bm(n, s2[p], d2[p], with_stats=True)
    assert a[0] == b[0] and b[1] == (a[1][0], 5, 50)


def test_networkx_triadic_census_agrees():
    nx = pytest.importorskip("networkx")
    for (n, s, d) in (graphgen.rmat(8, 16, 0.15, 1), graphgen.gnp(50, 0.1, 2), graphgen.chung_lu(500, 8, 2.1, 0.1, 4, 3)):
        G = nx.DiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(s.tolist(), d.tolist()))
        tc = nx.triadic_census(G)
        assert [tc[k] for k in oracle.CLASS_NAMES] == oracle.census_bm(n, s, d)


def test_golden_rmat_s10():
    """The scale-10 R-MAT census stored by tests/golden/make_golden.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "rmat_s10_r15_seed1.txt")
    vals = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    assert vals["n"] == n and vals["arcs"] == len(s)
    assert [vals[k] for k in oracle.CLASS_NAMES] == oracle.census_bm(n, s, d)

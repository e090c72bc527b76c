"""GPU parity: the census kernels through the C ABI against the CPU oracle, bit for bit.

Every case runs both kernel families (per-w union walk and bulk suffix counts) and, where
it matters, several tier settings, so that warp-tier vertices, CTA items and chunked hub
items are all exercised.  The tolerance is zero: counts are exact integers.
"""
import numpy as np
import pytest

import graphgen
import oracle
from census_facts import REVERSE, check_invariants, choose2, choose3, permute_classes

pytestmark = pytest.mark.gpu

ALGOS = [{"algo": 0}, {"algo": 1}, {"algo": 2}]
TIERS = [
    {},                                                       # defaults: warp <= 64, chunk 2048 / 4096
    {"warp_max_deg": 8, "chunk_entries": 512, "item_work": 2048},   # tiny chunks: hubs split
    {"warp_max_deg": 64, "chunk_entries": 8192, "item_work": 1 << 22, "ctas_per_sm": 1},
    {"map_mode": 2},                                          # no id map: every entry hashed
    {"warp_max_deg": 8, "chunk_entries": 512, "item_work": 2048, "map_mode": 2},
]


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_6308_gb300 import _build
    _build.build()
    import paper_1209_6308_gb300 as m
    m.load()
    return m


def gpu_census(tc, n, s, d, opts=None, device=False):
    import torch
    if device:
        s = torch.from_numpy(np.asarray(s, np.uint32).view(np.int32)).cuda()
        d = torch.from_numpy(np.asarray(d, np.uint32).view(np.int32)).cuda()
    with tc.Graph.from_arcs(n, s, d) as g:
        return g.census(options=opts)


def arcs(pairs):
    if not pairs:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    a = np.array(pairs, np.uint32)
    return a[:, 0].copy(), a[:, 1].copy()


# ------------------------------------------------------------------ configured workloads

@pytest.mark.parametrize("opts", [dict(a, **t) for a in ALGOS for t in TIERS])
def test_rmat_scale10_matches_oracle(tc, opts):
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    assert gpu_census(tc, n, s, d, opts) == oracle.census_bm(n, s, d)


def test_rmat_scale10_stats_match_oracle_cleaning(tc):
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    s2 = np.concatenate([s, s[:100], np.arange(7, dtype=np.uint32)])
    d2 = np.concatenate([d, d[:100], np.arange(7, dtype=np.uint32)])
    perm = np.random.default_rng(3).permutation(len(s2))
    c, st = oracle.census_bm(n, s2[perm], d2[perm], with_stats=True)
    with tc.Graph.from_arcs(n, s2[perm], d2[perm]) as g:
        info = g.stats()
        assert g.census() == c
    inv = oracle.invariants(n, s, d)
    assert (info["arcs"], info["loops_dropped"], info["dups_dropped"]) == st
    assert info["mutual"] == inv["M"] and info["e_sym"] == inv["M"] + inv["A"]


@pytest.mark.parametrize("algo", [0, 1, 2])
def test_chung_lu_golden(tc, algo):
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "chunglu_n5000_seed4_g11.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    n, s, d = graphgen.chung_lu(5000, 8.0, 2.1, 0.1, 4, 11)
    assert gpu_census(tc, n, s, d, {"algo": algo}) == [vals[k] for k in oracle.CLASS_NAMES]


@pytest.mark.parametrize("idx", range(6))
def test_chung_lu_batch_members_match_oracle(tc, idx):
    sizes = graphgen.loguniform_sizes(4096, 32, 65536, 4)
    i = int(np.argsort(sizes)[[0, 100, 1000, 2500, 4000, 4095][idx]])
    n, s, d = graphgen.chung_lu(int(sizes[i]), 8.0, 2.1, 0.1, 4, i)
    want = oracle.census_bm(n, s, d)
    for algo in (0, 1, 2):
        assert gpu_census(tc, n, s, d, {"algo": algo}) == want


# ------------------------------------------------------------------ brute force and closed forms

@pytest.mark.parametrize("seed", range(12))
def test_random_small_graphs_match_brute_force(tc, seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 65))
    n, s, d = graphgen.gnp(n, float(rng.choice([0.03, 0.1, 0.3, 0.7])), seed)
    want = oracle.census_brute(n, s, d)
    for opts in ({"algo": 0}, {"algo": 1}, {"algo": 1, "warp_max_deg": 2, "chunk_entries": 512}, {"algo": 2},
                 {"algo": 2, "warp_max_deg": 2, "chunk_entries": 512}):
        assert gpu_census(tc, n, s, d, opts, device=bool(seed % 2)) == want


def test_sampled_4_vertex_digraphs(tc):
    ordered = [(a, b) for a in range(4) for b in range(4) if a != b]
    rng = np.random.default_rng(11)
    for mask in rng.choice(1 << 12, 64, replace=False):
        s, d = arcs([ordered[i] for i in range(12) if mask >> i & 1])
        assert gpu_census(tc, 4, s, d) == oracle.census_brute(4, s, d), mask


@pytest.mark.parametrize("n", [3, 40, 150])
def test_complete_mutual_graph(tc, n):
    s, d = arcs([(a, b) for a in range(n) for b in range(n) if a != b])
    want = [0] * 16
    want[15] = choose3(n)
    for algo in (0, 1, 2):
        assert gpu_census(tc, n, s, d, {"algo": algo, "chunk_entries": 512, "warp_max_deg": 16}) == want


@pytest.mark.parametrize("n", [3, 50, 300])
def test_transitive_tournament(tc, n):
    s, d = arcs([(a, b) for a in range(n) for b in range(a + 1, n)])
    want = [0] * 16
    want[8] = choose3(n)
    for algo in (0, 1, 2):
        assert gpu_census(tc, n, s, d, {"algo": algo, "chunk_entries": 512, "warp_max_deg": 16}) == want


@pytest.mark.parametrize("n", [5, 70, 20000])
def test_hub_star_spans_many_chunks(tc, n):
    """A hub of degree n-1 > chunk: its list is split over CTA items."""
    s, d = arcs([(0, x) for x in range(1, n)])
    want = [0] * 16
    want[3] = choose2(n - 1)
    want[0] = choose3(n - 1)
    for algo in (0, 1, 2):
        assert gpu_census(tc, n, s, d, {"algo": algo, "chunk_entries": 1024}) == want
        assert gpu_census(tc, n, d, s, {"algo": algo, "chunk_entries": 1024}) == permute_classes(want, REVERSE)


def test_path_and_cycle(tc):
    n = 200
    s, d = arcs([(i, i + 1) for i in range(n - 1)])
    c = gpu_census(tc, n, s, d)
    assert c[5] == n - 2 and c[1] == (n - 1) * (n - 2) - 2 * (n - 2) and sum(c) == choose3(n)
    s, d = arcs([(0, 1), (1, 2), (2, 0)])
    want = [0] * 16
    want[9], want[1], want[0] = 1, 21, choose3(10) - 22
    assert gpu_census(tc, 10, s, d) == want


# ------------------------------------------------------------------ edge cases and errors

@pytest.mark.parametrize("n", [0, 1, 2, 3, 100])
def test_empty_graph(tc, n):
    s, d = arcs([])
    want = [0] * 16
    want[0] = choose3(n)
    assert gpu_census(tc, n, s, d) == want


def test_only_loops_and_duplicates(tc):
    s = np.array([3, 3, 5, 1, 1, 1], np.uint32)
    d = np.array([3, 3, 5, 2, 2, 2], np.uint32)
    with tc.Graph.from_arcs(8, s, d) as g:
        st = g.stats()
        c = g.census()
    assert (st["arcs"], st["loops_dropped"], st["dups_dropped"]) == (1, 3, 2)
    assert c == oracle.census_bm(8, s, d)


def test_out_of_range_id_is_an_error(tc):
    with pytest.raises(tc.TcError) as e:
        tc.Graph.from_arcs(5, np.array([0, 5], np.uint32), np.array([1, 2], np.uint32))
    assert e.value.status == tc.TC_ERR_RANGE


def test_too_many_vertices_is_an_error(tc):
    with pytest.raises(tc.TcError) as e:
        tc.Graph.from_arcs((1 << 30) + 1, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert e.value.status == tc.TC_ERR_RANGE


def test_bad_options_are_rejected(tc):
    n, s, d = graphgen.gnp(20, 0.2, 1)
    with tc.Graph.from_arcs(n, s, d) as g:
        for bad in ({"chunk_entries": 1000}, {"warp_max_deg": 4096}, {"algo": 7}, {"ctas_per_sm": 50},
                    {"algo": 2, "warp_max_deg": 256}, {"algo": 2, "chunk_entries": 16384}):
            with pytest.raises(tc.TcError):
                g.census(options=bad)
        with pytest.raises(tc.TcError):
            g.census(options={"schedule": 1})       # no cost model attached yet


# ------------------------------------------------------------------ CSR input and layout

def _csr_from_arcs(n, s, d):
    """Flagged symmetric CSR in the input ids, built here with numpy (test-side)."""
    fwd = set(zip(s.tolist(), d.tolist()))
    lists = [dict() for _ in range(n)]
    for a, b in fwd:
        if a == b:
            continue
        lists[a][b] = lists[a].get(b, 0) | 1
        lists[b][a] = lists[b].get(a, 0) | 2
    off = np.zeros(n + 1, np.uint64)
    adj = []
    for x in range(n):
        for y in sorted(lists[x]):
            adj.append((y << 2) | lists[x][y])
        off[x + 1] = len(adj)
    return off, np.array(adj, np.uint32)


def test_csr_input_matches_arc_input(tc):
    n, s, d = graphgen.rmat(9, 8, 0.2, 5)
    off, adj = _csr_from_arcs(n, s, d)
    with tc.Graph.from_csr(n, off, adj) as g:
        assert g.census() == oracle.census_bm(n, s, d)


def test_malformed_csr_is_rejected(tc):
    n, s, d = graphgen.gnp(30, 0.2, 2)
    off, adj = _csr_from_arcs(n, s, d)
    bad = adj.copy()
    bad[0] ^= 3 if bad[0] & 3 == 3 else 1          # break the mirrored direction bits
    for a in (bad, adj[::-1].copy()):
        with pytest.raises(tc.TcError) as e:
            tc.Graph.from_csr(n, off, a)
        assert e.value.status == tc.TC_ERR_ARG


def test_exported_csr_is_the_relabelled_graph(tc):
    n, s, d = graphgen.rmat(9, 8, 0.2, 6)
    with tc.Graph.from_arcs(n, s, d) as g:
        off, adj, perm = tc.tc_graph_export_csr(g.handle)
    assert sorted(perm.tolist()) == list(range(n))
    deg = np.diff(off.astype(np.int64))
    assert (deg[:-1] >= deg[1:]).all()                      # descending degree
    ref_off, ref_adj = _csr_from_arcs(n, perm[s], perm[d])
    assert (ref_off == off).all() and (ref_adj == adj).all()


# ------------------------------------------------------------------ other entry points

def test_async_census_into_device_tensor(tc):
    import torch
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with tc.Graph.from_arcs(n, s, d) as g:
        tc.tc_census_async(g.handle, out)
        torch.cuda.synchronize()
    c = [int(x) & ((1 << 64) - 1) for x in out.cpu().tolist()]
    c[0] = tc.tc_null_count(n, c)
    assert c == oracle.census_bm(n, s, d)


def test_batch_equals_individual(tc):
    gs, want = [], []
    for i, size in enumerate([40, 300, 2000, 9000]):
        n, s, d = graphgen.chung_lu(size, 8.0, 2.1, 0.1, 4, 100 + i)
        gs.append(tc.Graph.from_arcs(n, s, d))
        want.append(oracle.census_bm(n, s, d))
    assert tc.tc_census_batch([g.handle for g in gs]) == want
    for g in gs:
        g.close()


def test_repeated_census_is_stable(tc):
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    with tc.Graph.from_arcs(n, s, d) as g:
        first = g.census()
        for _ in range(5):
            assert g.census() == first
            assert g.census(options={"algo": 1}) == first


# ------------------------------------------------------------------ full-size workload

@pytest.fixture(scope="module")
def rmat20():
    return graphgen.rmat(20, 16, 0.2, 2)


def test_rmat_scale20_union_equals_suffix_and_tiers(tc, rmat20):
    n, s, d = rmat20
    with tc.Graph.from_arcs(n, s, d) as g:
        base = g.census(options={"algo": 1})
        assert g.census(options={"algo": 0}) == base
        assert g.census(options={"algo": 1, "chunk_entries": 1024, "warp_max_deg": 16}) == base
        assert g.census(options={"algo": 1, "map_mode": 2}) == base
        assert g.census(options={"algo": 0, "map_mode": 2}) == base
        assert g.census(options={"algo": 2}) == base
        assert g.census(options={"algo": 2, "chunk_entries": 512, "warp_max_deg": 16, "item_work": 4096}) == base
        inv_sum = sum(base)
    assert inv_sum == choose3(n)


def test_rmat_scale20_invariants(tc, rmat20):
    n, s, d = rmat20
    with tc.Graph.from_arcs(n, s, d) as g:
        c = g.census(options={"algo": 1})
    check_invariants(n, c, oracle.invariants(n, s, d))


def _induced(n, s, d, keep):
    idx = -np.ones(n, np.int64)
    idx[keep] = np.arange(len(keep))
    m = (idx[s] >= 0) & (idx[d] >= 0)
    return len(keep), idx[s[m]].astype(np.uint32), idx[d[m]].astype(np.uint32)


def test_rmat_scale20_random_induced_subgraph_matches_oracle(tc, rmat20):
    n, s, d = rmat20
    keep = np.sort(np.random.default_rng(20).choice(n, 50000, replace=False))
    k, ss, dd = _induced(n, s, d, keep)
    want = oracle.census_bm(k, ss, dd)
    for algo in (0, 1, 2):
        assert gpu_census(tc, k, ss, dd, {"algo": algo}) == want


def test_rmat_scale20_hub_core_matches_oracle(tc, rmat20):
    """The 1200 highest-degree vertices: the densest part, where hub chunks matter."""
    n, s, d = rmat20
    deg = np.bincount(s, minlength=n) + np.bincount(d, minlength=n)
    keep = np.sort(np.argsort(-deg, kind="stable")[:1200])
    k, ss, dd = _induced(n, s, d, keep)
    want = oracle.census_bm(k, ss, dd)
    for opts in ({"algo": 0}, {"algo": 1}, {"algo": 1, "chunk_entries": 512, "warp_max_deg": 4}, {"algo": 2},
                 {"algo": 2, "chunk_entries": 512, "warp_max_deg": 4}):
        assert gpu_census(tc, k, ss, dd, opts) == want


def test_page_locked_host_arcs_are_read_in_place(tc):
    """Arcs in page-locked host memory (read by the build's key kernel over the host link), in
    pageable host memory (copied first) and on the device give the same graph and census."""
    import torch
    n, s, d = graphgen.rmat(12, 16, 0.2, 21)
    s = np.concatenate([s, s[:100], np.arange(50, dtype=np.uint32)])   # repeats and loops
    d = np.concatenate([d, d[:100], np.arange(50, dtype=np.uint32)])
    want = oracle.census_bm(n, s, d)
    pin_s = torch.from_numpy(s.view(np.int32)).pin_memory()
    pin_d = torch.from_numpy(d.view(np.int32)).pin_memory()
    stats = []
    for src, dst in ((pin_s, pin_d), (s, d), (pin_s.cuda(), pin_d.cuda())):
        with tc.Graph(tc.tc_graph_create_arcs(n, src, dst), n) as g:
            assert g.census() == want
            st = g.stats()
            stats.append((st["e_sym"], st["arcs"], st["loops_dropped"], st["dups_dropped"]))
    assert stats[0] == stats[1] == stats[2]
    # one page-locked array and one pageable: the pageable one is copied
    with tc.Graph(tc.tc_graph_create_arcs(n, pin_s, d), n) as g:
        assert g.census() == want

"""The 64-state census on the GPU (Sec. 3, Fig. 2): per labelled state, the actors in increasing
vertex id of the caller's labels.  Compared state by state with the oracle (by definition on
small graphs, per linked pair on larger ones); tolerance zero."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


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


def gpu64(tc, n, s, d):
    with tc.Graph.from_arcs(n, s, d) as g:
        return g.census64()


def test_small_graphs_equal_the_definition(tc):
    rng = np.random.default_rng(21)
    ordered = [(a, b) for a in range(4) for b in range(4) if a != b]
    for mask in rng.choice(1 << 12, 40, replace=False):
        pairs = np.array([ordered[i] for i in range(12) if mask >> i & 1] or [(0, 1)], np.uint32)
        assert gpu64(tc, 4, pairs[:, 0], pairs[:, 1]) == oracle.census64_brute(4, pairs[:, 0], pairs[:, 1]), mask
    for n, p, seed in ((50, 0.2, 1), (120, 0.05, 2), (64, 0.5, 3)):
        n, s, d = graphgen.gnp(n, p, seed)
        assert gpu64(tc, n, s, d) == oracle.census64_brute(n, s, d)


def test_loops_duplicates_and_isolated_vertices(tc):
    s = np.array([3, 3, 7, 7, 7, 50, 2, 2], np.uint32)
    d = np.array([3, 7, 3, 3, 50, 7, 9, 9], np.uint32)
    assert gpu64(tc, 90, s, d) == oracle.census64_brute(90, s, d)
    empty = gpu64(tc, 10, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert empty[0] == 120 and sum(empty) == 120


@pytest.mark.parametrize("which", ["chunglu600", "rmat9", "star_and_clique", "tournament400"])
def test_skewed_graphs_equal_the_definition(tc, which):
    """By definition (every a < b < c) on the largest graphs the brute force covers quickly,
    chosen skewed so that hubs become CTA work items of the triangle walk (degree above 64)
    next to warp-tier vertices."""
    if which == "chunglu600":
        n, s, d = graphgen.chung_lu(600, 10.0, 2.1, 0.3, 7, 1)
    elif which == "rmat9":
        n, s, d = graphgen.rmat(9, 16, 0.25, 11)
    elif which == "star_and_clique":
        # a hub linked to everything one way or both, and a dense mutual block in the middle
        n = 500
        pairs = [(0, x) for x in range(1, n, 2)] + [(x, 0) for x in range(2, n, 3)]
        pairs += [(a, b) for a in range(200, 260) for b in range(200, 260) if a != b and (a * 7 + b) % 3]
        s = np.array([p[0] for p in pairs], np.uint32)
        d = np.array([p[1] for p in pairs], np.uint32)
    else:
        # a random tournament with a tenth of its pairs made mutual: every pair linked
        n = 400
        rng = np.random.default_rng(3)
        a, b = np.triu_indices(n, 1)
        flip = rng.random(len(a)) < 0.5
        both = rng.random(len(a)) < 0.1
        s0, d0 = np.where(flip, b, a), np.where(flip, a, b)
        s = np.concatenate([s0, d0[both]]).astype(np.uint32)
        d = np.concatenate([d0, s0[both]]).astype(np.uint32)
    want = oracle.census64_brute(n, s, d)
    with tc.Graph.from_arcs(n, s, d) as g:
        st = g.stats()
        got = g.census64()
    assert st["max_deg"] > 64
    assert got == want


def test_larger_graphs_equal_the_pair_route(tc):
    for n, s, d in (graphgen.rmat(10, 16, 0.15, 1), graphgen.chung_lu(5000, 12.0, 2.1, 0.1, 5, 4),
                    graphgen.rmat(13, 16, 0.2, 6)):
        assert gpu64(tc, n, s, d) == oracle.census64(n, s, d)


def test_fold_is_the_16_class_census(tc):
    n, s, d = graphgen.rmat(15, 16, 0.2, 9)
    table = tc.tc_tricode_table()
    with tc.Graph.from_arcs(n, s, d, options={"algo": 1}) as g:
        c64 = g.census64()
        c16 = g.census()
    fold = [0] * 16
    for state, k in enumerate(c64):
        fold[int(table[state])] += k
    assert fold == c16
    assert sum(c64) == n * (n - 1) * (n - 2) // 6


def test_csr_input_agrees(tc):
    from test_census_gpu import _csr_from_arcs
    n, s, d = graphgen.rmat(9, 8, 0.2, 5)
    off, adj = _csr_from_arcs(n, s, d)
    with tc.Graph.from_csr(n, off, adj) as g:
        assert g.census64() == oracle.census64_brute(n, s, d)

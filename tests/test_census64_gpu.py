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

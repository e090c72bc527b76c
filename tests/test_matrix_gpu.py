"""GPU parity of the matrix form of the census (tc_census_matrix: masked sums of products of the
bit-packed one-way, mutual and null dyad matrices; formulas pinned in test_matrix_formulas.py)
against the CPU oracle, count by count, tolerance zero.  Sizes cross the 64-column words and
the 64-row tiles raggedly, up to the largest n the call takes."""
import numpy as np
import pytest

import graphgen
import oracle
from census_facts import choose3

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


def mat(tc, n, s, d):
    with tc.Graph.from_arcs(n, s, d) as g:
        return g.census_matrix()


def test_every_three_vertex_digraph(tc):
    ordered = [(a, b) for a in range(3) for b in range(3) if a != b]
    for mask in range(64):
        pairs = [ordered[i] for i in range(6) if mask >> i & 1]
        s = np.array([p[0] for p in pairs], np.uint32)
        d = np.array([p[1] for p in pairs], np.uint32)
        assert mat(tc, 3, s, d) == oracle.census_brute(3, s, d), mask


@pytest.mark.parametrize("n,p", [(5, 0.5), (63, 0.1), (64, 0.3), (65, 0.05), (127, 0.2), (129, 0.6), (300, 0.02)])
def test_random_graphs_across_word_and_tile_edges(tc, n, p):
    n, s, d = graphgen.gnp(n, p, n)
    assert mat(tc, n, s, d) == oracle.census_bm(n, s, d)


def test_workload_graphs(tc):
    for (n, s, d) in (graphgen.rmat(10, 16, 0.15, 1), graphgen.rmat(12, 16, 0.2, 4),
                      graphgen.chung_lu(5000, 8.0, 2.1, 0.1, 4, 11)):
        assert mat(tc, n, s, d) == oracle.census_bm(n, s, d)


def test_closed_forms(tc):
    n = 100
    s, d = zip(*[(a, b) for a in range(n) for b in range(n) if a != b])
    want = [0] * 16
    want[15] = choose3(n)
    assert mat(tc, n, np.array(s, np.uint32), np.array(d, np.uint32)) == want
    n = 70
    s, d = zip(*[(a, b) for a in range(n) for b in range(a + 1, n)])
    want = [0] * 16
    want[8] = choose3(n)
    assert mat(tc, n, np.array(s, np.uint32), np.array(d, np.uint32)) == want
    for n in (0, 1, 2, 3, 10):
        want = [0] * 16
        want[0] = choose3(n)
        assert mat(tc, n, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) == want


def test_largest_size_agrees_with_the_oracle_and_the_kernels(tc):
    n, s, d = graphgen.rmat(14, 16, 0.2, 14)           # n = 2^14, the limit
    want = oracle.census_bm_parallel(n, s, d)
    with tc.Graph.from_arcs(n, s, d) as g:
        assert g.census_matrix() == want
        assert g.census(options={"algo": 2}) == want


def test_beyond_the_limit_is_a_range_error(tc):
    with tc.Graph.from_arcs((1 << 14) + 1, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as g:
        with pytest.raises(tc.TcError) as e:
            g.census_matrix()
        assert e.value.status == tc.TC_ERR_RANGE

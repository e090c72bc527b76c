"""Batched census (one persistent, graph-captured launch over many graphs) against the
per-graph census and the CPU oracle.  Counts are exact: tolerance zero."""
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


def _graphs(tc, specs):
    gs, arcs = [], []
    for (n, s, d) in specs:
        gs.append(tc.Graph.from_arcs(n, s, d))
        arcs.append((n, s, d))
    return gs, arcs


@pytest.fixture(scope="module")
def mixed(tc):
    specs = [graphgen.chung_lu(int(n), 8.0, 2.1, 0.1, 4, i) for i, n in enumerate([40, 33, 5000, 300, 20000, 2])]
    specs.append(graphgen.rmat(12, 16, 0.2, 9))
    specs.append((10, np.zeros(0, np.uint32), np.zeros(0, np.uint32)))     # no arcs
    gs, arcs = _graphs(tc, specs)
    yield gs, arcs
    for g in gs:
        g.close()


def test_batch_matches_oracle(tc, mixed):
    gs, arcs = mixed
    want = [oracle.census_bm(n, s, d) for (n, s, d) in arcs]
    assert tc.tc_census_batch([g.handle for g in gs]) == want
    for opts in ({"algo": 2}, {"algo": 2, "ctas_per_sm": 3, "chunk_entries": 1024, "item_work": 2048}):
        b = tc.tc_batch_create([g.handle for g in gs], options=opts)
        try:
            assert tc.tc_batch_census(b, len(gs)) == want, opts
            assert tc.tc_batch_census(b, len(gs)) == want, opts      # replays start from zero
        finally:
            tc.tc_batch_destroy(b)


def test_batch_object_replays_and_keeps_caller_order(tc, mixed):
    import torch
    gs, arcs = mixed
    want = [g.census() for g in gs]
    handles = [g.handle for g in gs][::-1]
    b = tc.tc_batch_create(handles)
    try:
        for _ in range(3):
            assert tc.tc_batch_census(b, len(handles)) == want[::-1]
        out = torch.zeros(16 * len(handles), dtype=torch.int64, device="cuda")
        tc.tc_batch_census_async(b, out)
        torch.cuda.synchronize()
        rows = out.cpu().numpy().astype(np.uint64).reshape(-1, 16)
        for i, w in enumerate(want[::-1]):
            assert [int(x) for x in rows[i][1:]] == w[1:]
    finally:
        tc.tc_batch_destroy(b)


def test_autotuned_plan_is_exact(tc, mixed):
    gs, arcs = mixed
    want = [g.census() for g in gs]
    b = tc.tc_batch_create([g.handle for g in gs])
    try:
        best, ms = tc.tc_batch_autotune(b, max_trials=6)
        assert ms > 0 and best["chunk_entries"] >= 512
        assert tc.tc_batch_census(b, len(gs)) == want
        # the whole coordinate descent: the default first, every trial timed, the best kept
        best, ms = tc.tc_batch_autotune(b)
        hist = tc.tc_batch_autotune_history(b)
        assert len(hist) > 6 and all(t > 0 for _, t in hist)
        assert ms == min(t for _, t in hist) and hist[0][1] >= ms
        assert {o["algo"] for o, _ in hist} == {0, 1, 2}
        assert {o["ctas_per_sm"] for o, _ in hist} >= {2, 3, 4, 6, 8}
        assert tc.tc_batch_census(b, len(gs)) == want
    finally:
        tc.tc_batch_destroy(b)


@pytest.mark.parametrize("algo", [0, 1, 2])
def test_batch_every_form(tc, mixed, algo):
    gs, arcs = mixed
    want = [g.census() for g in gs]
    b = tc.tc_batch_create([g.handle for g in gs], options={"algo": algo, "warp_max_deg": 8, "chunk_entries": 512})
    try:
        assert tc.tc_batch_census(b, len(gs)) == want
    finally:
        tc.tc_batch_destroy(b)


def test_chung_lu_batch_slice_matches_per_graph(tc):
    """512 graphs of the 4096-graph Chung-Lu batch workload (sizes log-uniform in [32, 65536])."""
    sizes = graphgen.loguniform_sizes(4096, 32, 65536, 4)
    idx = list(range(0, 4096, 8))
    gs = [tc.Graph.from_arcs(*graphgen.chung_lu(int(sizes[i]), 8.0, 2.1, 0.1, 4, i)) for i in idx]
    try:
        want = [g.census() for g in gs]
        assert tc.tc_census_batch([g.handle for g in gs]) == want
    finally:
        for g in gs:
            g.close()

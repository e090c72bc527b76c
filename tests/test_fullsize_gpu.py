"""GPU parity at the configured full sizes, against stored oracle results.

- The 4096 Chung-Lu graphs of the batched workload: every graph's 16 counts (null count
  included) against tests/golden/chunglu_batch4096_seed4.txt, written by the CPU oracle
  (tests/golden/make_golden.py), through the persistent batched launch (default and
  autotuned plans) and through the per-graph census in each kernel form.
- The R-MAT scale-20 workload: its 16 counts against tests/golden/rmat_s20_r20_seed2.txt
  (the oracle's OpenMP form of Fig. 5) in every kernel form, under the learned schedule, and
  as the sum of shards.
- The R-MAT scale-26 workload (the benchmark's), too large for the oracle's census: the two
  enumeration methods (per-pair walks and per-triangle) must agree count for count, and the
  census must meet the weighted-sum identities against the oracle's O(m) statistics.
Tolerance zero everywhere: the counts are exact integers."""
import os
import sys

import numpy as np
import pytest

import graphgen
import oracle
from census_facts import check_invariants

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
sys.path.insert(0, GOLDEN)
import make_golden  # noqa: E402


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


@pytest.fixture(scope="module")
def batch_graphs(tc):
    specs = graphgen.batch_chung_lu(4096, 32, 65536, 8.0, 2.1, 0.1, 4)
    gs = [tc.Graph.from_arcs(n, s, d, options={"algo": 1}) for (n, s, d) in specs]
    yield specs, gs
    for g in gs:
        g.close()


def test_batch_4096_golden_is_the_workload(batch_graphs):
    specs, _ = batch_graphs
    gold = make_golden.read_batch()
    assert len(gold) == 4096
    for (n, s, _), (gn, garcs, _) in zip(specs, gold):
        assert (n, len(s)) == (gn, garcs)


def test_batch_4096_persistent_launch_matches_oracle(tc, batch_graphs):
    _, gs = batch_graphs
    gold = make_golden.read_batch()
    want = [c for (_, _, c) in gold]
    got = tc.tc_census_batch([g.handle for g in gs])
    bad = [i for i, (a, b) in enumerate(zip(got, want)) if a != b]
    assert not bad, f"{len(bad)} graphs differ, first {bad[:5]}"
    for opts in ({"algo": 1}, {"algo": 2}):
        b = tc.tc_batch_create([g.handle for g in gs], options=opts)
        try:
            assert tc.tc_batch_census(b, len(gs)) == want, opts
            tc.tc_batch_autotune(b, max_trials=8)
            assert tc.tc_batch_census(b, len(gs)) == want, opts
        finally:
            tc.tc_batch_destroy(b)


@pytest.mark.parametrize("algo", [0, 1, 2])
def test_batch_4096_per_graph_census_matches_oracle(tc, batch_graphs, algo):
    _, gs = batch_graphs
    gold = make_golden.read_batch()
    bad = [i for i, (g, (_, _, c)) in enumerate(zip(gs, gold)) if g.census(options={"algo": algo}) != c]
    assert not bad, f"{len(bad)} graphs differ, first {bad[:5]}"


@pytest.fixture(scope="module")
def rmat20():
    return graphgen.rmat(20, 16, 0.2, 2)


def _s20_golden():
    path = os.path.join(GOLDEN, make_golden.S20_FILE)
    if not os.path.exists(path):
        pytest.skip("scale-20 oracle fixture not written")
    return make_golden.read_counts(make_golden.S20_FILE)


def test_rmat20_every_form_matches_oracle(tc, rmat20):
    gn, garcs, want = _s20_golden()
    n, s, d = rmat20
    assert (n, len(s)) == (gn, garcs)
    with tc.Graph.from_arcs(n, s, d, options={"algo": 1}) as g:
        for opts in ({"algo": 1}, {"algo": 2}, {"algo": 1, "map_mode": 2},
                     {"algo": 2, "ctas_per_sm": 3, "chunk_entries": 4096}):
            assert g.census(options=opts) == want, opts
    with tc.Graph.from_arcs(n, s, d) as g:                 # the union walk is the graph's default form
        assert g.census() == want


def test_rmat20_shards_match_oracle(tc, rmat20):
    import torch
    from paper_1209_6308_gb300 import shard
    _, _, want = _s20_golden()
    n, s, d = rmat20
    with tc.Graph.from_arcs(n, s, d, options={"algo": 1}) as g:
        for opts, world in (({"algo": 2}, 4), ({"algo": 1}, 3)):
            total = torch.zeros(16, dtype=torch.int64, device="cuda")
            out = torch.zeros(16, dtype=torch.int64, device="cuda")
            for r in range(world):
                tc.tc_census_shard(g.handle, out, r, world, options=opts)
                total += out
            torch.cuda.synchronize()
            assert shard.census_of_sum(n, total.cpu()) == want, (opts, world)


@pytest.fixture(scope="module")
def small_model(tc):
    """A cost model trained briefly on two small R-MAT graphs, per kernel form: its quality does
    not matter here, only that the learned plans it makes give the oracle's counts."""
    from paper_1209_6308_gb300 import learned
    models = {}
    for algo in (1, 2):
        models[algo], _ = learned.train_cost_model(scales=(13, 14), steps=60, options={"algo": algo})
    yield models
    for m in models.values():
        tc.tc_costmodel_destroy(m)


def test_rmat20_learned_schedule_matches_oracle(tc, rmat20, small_model):
    from paper_1209_6308_gb300 import learned
    _, _, want = _s20_golden()
    n, s, d = rmat20
    for algo, model in small_model.items():
        with tc.Graph.from_arcs(n, s, d, options={"algo": algo}) as g:
            learned.attach(model, g)
            assert g.census(options={"algo": algo, "schedule": 1}) == want, algo


@pytest.mark.parametrize("which", ["rmat13", "hubcore20"])
def test_learned_schedule_matches_oracle_on_graphs_with_hub_items(tc, small_model, rmat20, which):
    """The learned schedule against the oracle's own census (not against the plain GPU
    schedule), on graphs whose hubs become several CTA items and span several chunks."""
    from paper_1209_6308_gb300 import learned
    if which == "rmat13":
        n, s, d = graphgen.rmat(13, 16, 0.2, 5)
    else:
        n0, s0, d0 = rmat20
        deg = np.bincount(s0, minlength=n0) + np.bincount(d0, minlength=n0)
        keep = np.sort(np.argsort(-deg, kind="stable")[:1200])
        idx = -np.ones(n0, np.int64)
        idx[keep] = np.arange(len(keep))
        m = (idx[s0] >= 0) & (idx[d0] >= 0)
        n, s, d = len(keep), idx[s0[m]].astype(np.uint32), idx[d0[m]].astype(np.uint32)
    want = oracle.census_bm(n, s, d)
    for algo, model in small_model.items():
        for extra in ({}, {"chunk_entries": 512, "warp_max_deg": 8, "item_work": 2048}):
            with tc.Graph.from_arcs(n, s, d, options={"algo": algo}) as g:
                learned.attach(model, g)
                assert g.census(options=dict({"algo": algo, "schedule": 1}, **extra)) == want, (algo, extra)


def test_rmat26_methods_agree_and_meet_the_identities(tc):
    """The benchmark's workload: per-pair walks (suffix form) and per-triangle enumeration give
    the same 16 counts, which meet every O(m) weighted-sum identity of the oracle's statistics
    (the triangle count, superlinear, is left to the smaller fixtures)."""
    n, s, d = graphgen.rmat(26, 16, 0.2, 3)
    with tc.Graph.from_arcs(n, s, d, options={"algo": 2}) as g:
        tri = g.census(options={"algo": 2})
        suf = g.census(options={"algo": 1})
    assert tri == suf
    inv = oracle.invariants(n, s, d, triangles=False)
    check_invariants(n, tri, inv, triangles=False)

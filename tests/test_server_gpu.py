"""Census serving (continuous batching of requests into wave launches of the census kernel):
every request's counts equal the graph's own census, however its work was sliced and mixed
with other requests; memory admission refuses what does not fit; host-side errors are
reported, not hung.  Counts are exact: tolerance zero."""
import threading

import numpy as np
import pytest

import graphgen
import oracle
from census_facts import check_invariants

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


SUFFIX = {"algo": 1}


@pytest.fixture(scope="module")
def pool(tc):
    """Graphs of very different sizes (hub items, warp-tier blocks, empty and tiny cases), each
    with its census, checked against the oracle."""
    specs = [graphgen.chung_lu(int(n), 12.0, 2.1, 0.1, 5, i) for i, n in enumerate([1000, 47, 20000, 3, 150000])]
    specs.append(graphgen.rmat(12, 16, 0.15, 1))
    specs.append(graphgen.rmat(16, 16, 0.2, 16))
    specs.append((10, np.zeros(0, np.uint32), np.zeros(0, np.uint32)))
    specs.append(graphgen.gnp(60, 0.3, 3))
    gs = [tc.Graph.from_arcs(n, s, d, options=SUFFIX) for (n, s, d) in specs]
    # every served result is compared with the oracle's census of its graph; the 150,000-vertex
    # graph, minutes for the oracle, is pinned by the weighted-sum identities of the oracle's
    # statistics (triangles included) and the agreement of the per-pair and per-triangle forms
    want = []
    for (n, s, d), g in zip(specs, gs):
        c = g.census(options=SUFFIX)
        if len(s) < 1500000:
            assert c == oracle.census_bm_parallel(n, s, d)
        else:
            assert g.census(options={"algo": 2}) == c
            check_invariants(n, c, oracle.invariants(n, s, d))
        want.append(c)
    yield gs, want, specs
    for g in gs:
        g.close()


def _serve(tc, gs, order, options=None, census=None, threads=1):
    with tc.Server(options, census or SUFFIX) as srv:
        ids = [srv.add(g) for g in gs]
        rid_graph = {}
        lock = threading.Lock()

        def submit(part):
            for k in part:
                r = srv.submit(ids[k])
                with lock:
                    rid_graph[r] = k

        parts = [order[t::threads] for t in range(threads)]
        ts = [threading.Thread(target=submit, args=(p,)) for p in parts]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        srv.drain(120000)
        res = srv.poll(len(order) + 1)
        stats = srv.stats()
    return res, rid_graph, ids, stats


def test_oracle_agrees_with_the_standalone_census_on_small_pool_graphs(tc, pool):
    gs, want, specs = pool
    for k, (n, s, d) in enumerate(specs):
        if len(s) <= 40000:
            assert want[k] == oracle.census_bm(n, s, d), k


@pytest.mark.parametrize("form", [1, 2])
def test_mixed_requests_equal_standalone_census(tc, pool, form):
    gs, want, _ = pool
    rng = np.random.default_rng(11)
    order = list(rng.integers(0, len(gs), 300))
    # a short quantum forces large censuses into many slices shared with other requests
    res, rid_graph, ids, stats = _serve(tc, gs, order, {"quantum_us": 40, "lanes": 2}, census={"algo": form})
    assert len(res) == len(order)
    assert stats["completed"] == len(order) and stats["error"] == 0
    for r in res:
        k = rid_graph[r.id]
        assert r.status == 0
        assert r.graph == ids[k]
        assert r.census() == want[k], (k, r.waves)
        assert r.submit_ns <= r.start_ns <= r.done_ns
    assert max(r.waves for r in res) > 1          # slicing happened
    assert stats["slices"] > stats["waves"]        # waves mixed requests


@pytest.mark.parametrize("lanes,quantum,form", [(1, 1000, 1), (4, 200, 1), (3, 5, 1), (1, 1000, 2), (3, 5, 2)])
def test_lane_and_quantum_settings_keep_counts(tc, pool, lanes, quantum, form):
    gs, want, _ = pool
    order = [k % len(gs) for k in range(3 * len(gs))]
    res, rid_graph, _, stats = _serve(tc, gs, order, {"quantum_us": quantum, "lanes": lanes}, census={"algo": form})
    assert sorted(rid_graph) == sorted(r.id for r in res)
    for r in res:
        assert r.census() == want[rid_graph[r.id]]
        assert r.lane < lanes


def test_split_work_items_keep_counts(tc, pool):
    """A tiny item cap cuts every hub item into many pair ranges (each restaging N[u])."""
    gs, want, _ = pool
    order = list(range(len(gs))) * 2
    for form in (1, 2):
        res, rid_graph, ids, _ = _serve(tc, gs, order, {"quantum_us": 200, "max_item_units": 1}, census={"algo": form})
        for r in res:
            assert r.census() == want[rid_graph[r.id]], form
    with tc.Server({"max_item_units": 1}, SUFFIX) as srv, tc.Server(None, SUFFIX) as ref:
        gid, rid = srv.add(gs[6]), ref.add(gs[6])             # R-MAT scale 16
        split_items = tc.tc_server_graph_units(srv.handle, gid)[1]
        plain_items = tc.tc_server_graph_units(ref.handle, rid)[1]
        assert split_items > plain_items


def test_union_kernel_server(tc, pool):
    gs, want, _ = pool
    order = list(range(len(gs))) * 2
    res, rid_graph, _, _ = _serve(tc, gs, order, {"quantum_us": 100}, census={"algo": 0})
    for r in res:
        assert r.census() == want[rid_graph[r.id]]


def test_submits_from_several_threads(tc, pool):
    gs, want, _ = pool
    rng = np.random.default_rng(12)
    order = list(rng.integers(0, len(gs), 400))
    res, rid_graph, _, _ = _serve(tc, gs, order, {"quantum_us": 100, "max_active": 16}, threads=4)
    assert len(res) == len(order)
    for r in res:
        assert r.census() == want[rid_graph[r.id]]


def test_learned_schedule_server(tc, pool):
    gs, want, _ = pool
    model = tc.tc_costmodel_create(3)
    try:
        tc.tc_costmodel_set_norm(model, np.ones(4, np.float32), np.ones(4, np.float32), 8.0, 1.0)
        for g in gs:
            tc.tc_graph_attach_costmodel(g.handle, model)
        order = list(range(len(gs))) * 3
        for form in (1, 2):
            res, rid_graph, _, _ = _serve(tc, gs, order, {"quantum_us": 100},
                                          census={"algo": form, "schedule": tc.TC_SCHED_LEARNED})
            for r in res:
                assert r.census() == want[rid_graph[r.id]], form
    finally:
        tc.tc_costmodel_destroy(model)


def test_learned_server_refuses_a_graph_without_a_model(tc):
    n, s, d = graphgen.chung_lu(5000, 12.0, 2.1, 0.1, 5, 99)
    with tc.Graph.from_arcs(n, s, d) as g, tc.Server(None, {"algo": 1, "schedule": tc.TC_SCHED_LEARNED}) as srv:
        with pytest.raises(tc.TcError) as e:
            srv.add(g)
        assert e.value.status == tc.TC_ERR_ARG


def test_memory_admission(tc, pool):
    gs, want, _ = pool
    small, big = gs[0], gs[6]                          # 1000-vertex Chung-Lu, R-MAT scale 16
    with tc.Server(None, SUFFIX) as probe:
        a = probe.add(small)
        need_small = probe.stats()["resident_bytes"]
        probe.remove(a)
        assert probe.stats()["resident_bytes"] == 0
    with tc.Server({"budget_bytes": need_small + 1024}, SUFFIX) as srv:
        gid = srv.add(small)
        with pytest.raises(tc.TcError) as e:
            srv.add(big)
        assert e.value.status == tc.TC_ERR_OOM
        st = srv.stats()
        assert st["refused"] == 1 and st["graphs"] == 1 and st["resident_bytes"] == need_small
        for _ in range(5):
            srv.submit(gid)
        srv.drain(60000)
        res = srv.poll(10)
        assert [r.census() for r in res] == [want[0]] * 5
        srv.remove(gid)
        with pytest.raises(tc.TcError):
            srv.add(big)                                # still larger than the whole budget


def test_host_side_errors(tc, pool):
    gs, _, _ = pool
    with tc.Server({"max_pending": 4, "quantum_us": 20}, SUFFIX) as srv:
        with pytest.raises(tc.TcError) as e:
            srv.submit(12345)
        assert e.value.status == tc.TC_ERR_ARG
        gid = srv.add(gs[6])
        rids = [srv.submit(gid) for _ in range(4)]
        # requests in the server hold their graph
        with pytest.raises(tc.TcError) as e:
            srv.remove(gid)
        assert e.value.status == tc.TC_ERR_BUSY
        srv.drain(60000)
        assert sorted(r.id for r in srv.poll(10)) == sorted(rids)
        srv.remove(gid)
        with pytest.raises(tc.TcError) as e:
            srv.remove(gid)
        assert e.value.status == tc.TC_ERR_ARG


def test_poll_times_out_and_drain_of_an_idle_server(tc):
    with tc.Server(None, SUFFIX) as srv:
        assert srv.poll(4, timeout_ms=20) == []
        srv.drain(10)

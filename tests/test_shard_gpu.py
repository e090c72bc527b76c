"""GPU parity of the sharded census (paper Sec. 6-7: the connected pairs (u, v) are independent,
so the census is the sum over any partition of them).  On one GPU the shards of a world of W
ranks run one after another through the C ABI (tc_census_shard); their counters summed, with
the null count taken from the sum, must equal the CPU oracle's census exactly, for several W,
kernel forms and tier settings, including worlds larger than the number of work units."""
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


def shard_sum(tc, g, n, world, opts=None):
    """Every rank's shard run in turn; the summed counters and the shards' own counts."""
    import torch
    from paper_1209_6308_gb300 import shard
    total = torch.zeros(16, dtype=torch.int64, device="cuda")
    parts = []
    for r in range(world):
        out = torch.full((16,), 3, dtype=torch.int64, device="cuda")     # must be overwritten
        tc.tc_census_shard(g.handle, out, r, world, options=opts)
        torch.cuda.synchronize()
        parts.append(out.cpu())
        total += out
    return shard.census_of_sum(n, total.cpu()), parts


GRAPHS = {
    "rmat10": lambda: graphgen.rmat(10, 16, 0.15, 1),
    "rmat13": lambda: graphgen.rmat(13, 16, 0.2, 5),
    "chunglu20k": lambda: graphgen.chung_lu(20000, 8.0, 2.1, 0.1, 4, 3),
}
OPTS = [
    {"algo": 1},
    {"algo": 0},
    {"algo": 1, "warp_max_deg": 8, "chunk_entries": 512, "item_work": 2048},   # many items, chunked hubs
    {"algo": 1, "map_mode": 2},
    {"algo": 2},
    {"algo": 2, "warp_max_deg": 8, "chunk_entries": 512, "item_work": 2048},
]


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("opts", OPTS)
def test_shards_sum_to_the_oracle_census(tc, name, opts):
    n, s, d = GRAPHS[name]()
    want = oracle.census_bm(n, s, d)
    with tc.Graph.from_arcs(n, s, d) as g:
        assert g.census(options=opts) == want
        for world in (1, 2, 3, 7):
            got, parts = shard_sum(tc, g, n, world, opts)
            assert got == want, world
            assert all(int(p[0]) == 0 for p in parts)


def test_more_ranks_than_work_units(tc):
    """A small graph over 500 ranks: most shards are empty (their counters all zero), and the
    sum is still the census."""
    n, s, d = graphgen.gnp(60, 0.1, 4)
    want = oracle.census_bm(n, s, d)
    with tc.Graph.from_arcs(n, s, d) as g:
        got, parts = shard_sum(tc, g, n, 500)
        assert got == want
        assert sum(1 for p in parts if int(p.abs().sum()) == 0) > 400


def test_shard_bounds_cover_the_work_once(tc):
    n, s, d = graphgen.rmat(13, 16, 0.2, 5)
    opts = {"algo": 1, "warp_max_deg": 8, "chunk_entries": 512, "item_work": 2048}
    with tc.Graph.from_arcs(n, s, d) as g:
        one = tc.tc_census_shard_bounds(g.handle, 1, options=opts)
        (i0, v0), (ni, v_end) = one
        assert i0 == 0 and ni > 0 and v_end > v0
        for world in (2, 5, 16):
            b = tc.tc_census_shard_bounds(g.handle, world, options=opts)
            assert b.shape == (world + 1, 2)
            assert tuple(b[0]) == (0, v0) and tuple(b[-1]) == (ni, v_end)
            assert np.all(np.diff(b[:, 0].astype(np.int64)) >= 0)
            assert np.all(np.diff(b[:, 1].astype(np.int64)) >= 0)
            # a shard that starts inside the warp tier has no items left
            for r in range(world + 1):
                if b[r, 1] > v0:
                    assert b[r, 0] == ni


def test_empty_and_edgeless_graphs(tc):
    import torch
    for n in (0, 1, 5):
        with tc.Graph.from_arcs(n, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as g:
            got, _ = shard_sum(tc, g, n, 3)
            assert got == oracle.census_bm(n, np.zeros(0, np.uint32), np.zeros(0, np.uint32))


def test_bad_rank_or_world_is_an_argument_error(tc):
    import torch
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with tc.Graph.from_arcs(n, s, d) as g:
        for rank, world in ((2, 2), (0, 0), (5, 3)):
            with pytest.raises(tc.TcError) as e:
                tc.tc_census_shard(g.handle, out, rank, world)
            assert e.value.status == tc.TC_ERR_ARG

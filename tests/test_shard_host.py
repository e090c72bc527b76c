"""Host side of the sharded census (paper Sec. 6-7: the census is the sum over any partition of
the connected pairs), with world_size 2 over gloo on the CPU: each rank takes a share of the
pairs, the ranks sum their 16 counters with the same call the NCCL ranks of the benchmark make,
and the null count is taken from the sum in 128-bit.  The shares here are the CPU oracle's
vertex samples (u = rank mod world), so the test needs no GPU; the result must equal the
oracle's whole census exactly."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, graph, out):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1209_6308_gb300 import shard
    n, s, d = graph
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        og = oracle.SampledGraph(n, s, d)
        _, part, _, _ = og.sample(world, rank)       # pairs (u, v) with u = rank (mod world)
        og.close()
        counts = torch.tensor([0] + [int(x) for x in part[1:]], dtype=torch.int64)
        shard.allreduce_counts(dist, counts)
        out.put((rank, shard.census_of_sum(n, counts)))
    finally:
        dist.destroy_process_group()


def _run(world, graph):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, graph, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sum_equals_the_oracle_census(world):
    import graphgen
    import oracle
    n, s, d = graphgen.rmat(10, 16, 0.15, 1)
    want = oracle.census_bm(n, s, d)
    res = _run(world, (n, s, d))
    assert sorted(res) == list(range(world))
    for r, got in res.items():
        assert got == want, r


def test_null_count_of_the_sum_needs_128_bits():
    """At n = 2^26 the null count exceeds 2^64: the sum of the shards' counters stays in uint64
    and the null count is taken in 128-bit from C(n,3)."""
    from paper_1209_6308_gb300 import shard
    n = 1 << 26
    counts = np.zeros(16, np.int64)
    counts[1] = 5
    counts[2] = 7
    got = shard.census_of_sum(n, counts)
    total = n * (n - 1) * (n - 2) // 6
    assert total > 1 << 64
    assert got[0] == total - 12 and got[1:3] == [5, 7]

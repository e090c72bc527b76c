"""Census sharded over the ranks of a process group (paper Sec. 6-7: the connected pairs of
Fig. 5 step 2.1 are independent, so the census is the sum of any partition of them).

Every rank holds the same graph and runs its shard through ``tc_census_shard`` (C ABI); the
only exchange is one sum of the shards' 16 counters (an all-reduce of 128 bytes), after which
the null count C(n,3) - sum is taken on the host in 128-bit arithmetic (``tc_null_count``,
Fig. 5 steps 3-5).  This module only sequences those calls: the census itself runs in the
library's kernels.
"""
from __future__ import annotations

from . import tc_census_shard, tc_null_count

_MASK64 = (1 << 64) - 1


def allreduce_counts(dist, counts) -> None:
    """Sum a 16-element int64 tensor of per-shard counters over every rank, in place.  The
    counters are uint64 held in int64: a two's-complement sum wraps like the unsigned one."""
    if dist is not None:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM)


def census_of_sum(n: int, counts) -> list:
    """The 16-class census from the summed counters of classes 1..15: index 0 becomes the null
    count C(n,3) minus the rest (128-bit, on the host)."""
    c = [int(x) & _MASK64 for x in (counts.tolist() if hasattr(counts, "tolist") else counts)]
    c[0] = 0
    c[0] = tc_null_count(n, c)
    return c


def enqueue_shard(g, d_out16, rank: int, world: int, stream=None, options=None) -> None:
    """This rank's share of the census of g into d_out16 (16 uint64 on the device)."""
    tc_census_shard(g.handle if hasattr(g, "handle") else g, d_out16, rank, world, stream=stream, options=options)


def sharded_census(g, n: int, d_out16, rank: int, world: int, dist=None, stream=None, options=None) -> list:
    """Run this rank's shard, sum the counters over the process group and return the full
    census (every rank gets it).  With dist None and world 1 this is the plain census."""
    enqueue_shard(g, d_out16, rank, world, stream=stream, options=options)
    if dist is not None and stream is not None:
        # the collective runs on torch's current stream: make it the census's stream
        import torch
        s = stream if isinstance(stream, torch.cuda.Stream) else torch.cuda.ExternalStream(int(stream))
        with torch.cuda.stream(s):
            allreduce_counts(dist, d_out16)
    else:
        allreduce_counts(dist, d_out16)
    return census_of_sum(n, d_out16.cpu())

"""Host logic of bench.py that needs no GPU: the multi-rank reduction (world_size 2 over gloo
on the CPU, the same calls the NCCL ranks make), the whole-job value, the command-line
defaults, and the reference arm's behaviour on ranks other than 0."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(dist, times[rank], "cpu")
        out.put((rank, ms, bench.job_value(1000, ms)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 40.0]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 40.0                      # every rank sees the slowest rank's time
        assert value == pytest.approx(1000 / 0.040)   # one census's arcs: the ranks shard it


def test_single_process_reduction_is_the_identity():
    import bench
    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25
    assert bench.job_value(500, 2.0) == pytest.approx(250000.0)


def test_defaults_finish_in_minutes(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and 1 <= a.steps <= 20
    assert a.impl == "ours" and a.serve_seconds == 60.0 and bench.WORKLOAD["scale"] == 26


@pytest.mark.parametrize("argv,scale", [([], 26), (["--scale", "20"], 20), (["--scale", "10"], 10), ([], 26)])
def test_workload_follows_the_scale_option(monkeypatch, argv, scale):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    bench.parse()
    assert bench.WORKLOAD["scale"] == scale
    assert bench.WORKLOAD == bench.WORKLOADS[scale] and bench.WORKLOAD is not bench.WORKLOADS[scale]
    assert bench.WORKLOADS[20]["name"] == "rmat20_ef16_r20_seed2"


def test_reference_arm_on_other_ranks_exits_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    called = []
    monkeypatch.setattr(bench, "workload", lambda: called.append(1))
    assert bench.run_reference(bench.parse()) == 0
    assert not called


def test_bytes_alg_follows_the_scope_formula():
    """8(n+1) + 8 E + sum over upper pairs (4 d_v + 16) + 128, from the graph's statistics."""
    import bench
    info = {"e_sym": 10, "sum_dv_upper": 37}
    assert bench.bytes_alg_8d(5, info) == 8 * 6 + 8 * 10 + 4 * 37 + 16 * 10 + 128


def test_census_code_hash_ignores_comments_only():
    """The stored DRAM traffic stays valid across comment edits of the kernel's source, not code
    edits; the committed capture of the triangle walk at scale 26 names its hash and bytes."""
    import bench
    src = "int a = 1; // one\n/* block\n comment */\n\nint b = 2;\n"
    same = "// header\nint a = 1;\n\nint b = 2;   \n"
    other = "int a = 1;\nint b = 3;\n"
    assert bench.census_code_hash(src) == bench.census_code_hash(same)
    assert bench.census_code_hash(src) != bench.census_code_hash(other)
    with open(bench.traffic_file("rmat26_ef16_r20_seed3", "k_triangles")) as f:
        kv = dict(line.split(":", 1) for line in f if ":" in line and not line.startswith("#"))
    assert "code_sha256_16" in kv and float(kv["dram_bytes_per_launch"]) > 0

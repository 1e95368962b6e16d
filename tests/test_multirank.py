"""The N > 1 host path of the benchmark on CPU: world_size-2 gloo ranks
(the benchmark runs one independent replica per GPU, no data-path
collective; the ranks only agree on the slowest rank's time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # every rank reports its own step time; all of them get the slowest
        t = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
        assert bench.dist_env() == (ws, rank, rank)
        out.put((rank, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = dict(q.get(timeout=5) for _ in range(ws))
    assert got == {0: 15.0, 1: 15.0}


def test_whole_job_value_counts_every_replica():
    # 64 BFS of 128.3M edges in 10 ms on each of N replicas: N times one replica's rate
    one = bench.whole_job_gteps(1, 64, 128_304_424, 0.010)
    assert one == pytest.approx(64 * 128_304_424 / 0.010 / 1e9)
    assert bench.whole_job_gteps(4, 64, 128_304_424, 0.010) == pytest.approx(4 * one)
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_reference_arm_prints_only_on_rank_zero(capsys, monkeypatch):
    """Under torchrun the other ranks of the reference arm exit without work."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "ref_sources": 1, "gpus": 2})()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


def test_traffic_record_needs_the_same_code_and_threshold(tmp_path):
    """The bench reports a kernel's DRAM bytes only from a capture of the same
    code (a digest of its sources without comments) at the same push/pull
    threshold."""
    src = tmp_path / "k.cu"
    src.write_text("// a comment\n__global__ void k() { int x = 1; }\n")
    dig = bench.code_digest(["k.cu"], root=str(tmp_path))
    prof = tmp_path / "p.md"
    prof.write_text(f"traffic-record: kernel=k digest={dig} beta=24 bytes_per_launch=1000 launches=64\n"
                    f"traffic-record: kernel=k digest={dig} beta=16 bytes_per_launch=900 launches=64\n")
    old_root = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        assert bench.recorded_traffic("p.md", ["k.cu"], 24) == 1000.0
        assert bench.recorded_traffic("p.md", ["k.cu"], 16) == 900.0
        assert bench.recorded_traffic("p.md", ["k.cu"], 8) is None
        src.write_text("// another comment\n__global__ void k() { int x = 1; }\n")   # comments do not count
        assert bench.recorded_traffic("p.md", ["k.cu"], 24) == 1000.0
        src.write_text("__global__ void k() { int x = 2; }\n")                        # code does
        assert bench.recorded_traffic("p.md", ["k.cu"], 24) is None
    finally:
        bench.ROOT = old_root


def test_traffic_record_of_a_sample_scales_by_algorithmic_bytes(tmp_path):
    """A record taken on a sample of the sources, with the tile shape it ran
    and the sample's mean algorithmic bytes, is scaled to the bench's mean
    algorithmic bytes, and matches only its own shape."""
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    dig = bench.code_digest(["k.cu"], root=str(tmp_path))
    (tmp_path / "p.md").write_text(
        f"traffic-record: kernel=k digest={dig} beta=16 shape=1,4 bytes_per_launch=150 alg_per_launch=100 "
        f"launches=8\n")
    old_root = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        assert bench.recorded_traffic("p.md", ["k.cu"], 16, "1,4", 110.0) == pytest.approx(165.0)
        assert bench.recorded_traffic("p.md", ["k.cu"], 16, "1,4") == 150.0
        assert bench.recorded_traffic("p.md", ["k.cu"], 16, "2,0", 110.0) is None
    finally:
        bench.ROOT = old_root


def test_committed_bfs_traffic_records_match_the_committed_kernel():
    """The DRAM traffic the bench reports beside k_bfs comes from records in
    the kernel's profile summary that were captured on the same kernel code
    (their digest equals that of the BFS sources as committed) at the tile
    shape the autotuner picks on the benchmark graph, for each threshold it
    picks there; a kernel change without a new capture fails here."""
    for beta in (16, 20, 24):
        t = bench.recorded_traffic(bench.BFS_PROFILE, bench.BFS_KERNEL_SOURCES, beta, "1,0", 101.3e6)
        assert t is not None, beta
        assert 1.3 < t / 101.3e6 < 1.7      # the 32-byte pull records: ~1.5x the algorithmic bytes

"""Host-side logic of bench.py: the max-over-ranks reduction across two gloo ranks on CPU,
the ncu-summary reader and the argument defaults (no GPU)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v = bench.reduce_max(10.0 + rank * 5.0, world, dist)
    q.put((rank, v))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 15.0), (1, 15.0)]


def test_counters_are_null_when_kernel_changed(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "s.md"
    body = "- traffic_bytes_per_ray: 123.0\n- l2_bytes_per_ray: 700\n- l2_frac: 0.45\n- issue_frac: 0.66\n"
    f.write_text("- kernel_source_hash: 0000\n" + body)
    monkeypatch.setattr(bench, "NCU_SUMMARY", {2: str(f)})
    assert bench.read_counters(2) == {}
    assert bench.read_counters(1) == {}  # the persistent form has no per-kernel summary
    f.write_text(f"- kernel_source_hash: {bench.source_hash(bench.TRAVERSE_SOURCES[2])}\n" + body)
    assert bench.read_counters(2) == {"traffic_bytes_per_ray": 123.0, "l2_bytes_per_ray": 700.0, "l2_frac": 0.45,
                                      "issue_frac": 0.66}


def test_committed_traversal_summary_matches_the_sources():
    """The committed ncu summary of the benchmarked traversal kernel was taken on the current
    sources (otherwise the bench reports its DRAM / L2 counters as null)."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.read_counters(2)
    assert set(c) == {"traffic_bytes_per_ray", "l2_bytes_per_ray", "l2_frac", "issue_frac"}

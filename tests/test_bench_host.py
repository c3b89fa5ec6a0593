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


def test_traffic_is_null_when_kernel_changed(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "s.md"
    f.write_text("- kernel_source_hash: 0000\n- traffic_bytes_per_ray: 123.0\n")
    monkeypatch.setattr(bench, "NCU_SUMMARY", {2: str(f)})
    assert bench.read_traffic(2) is None
    assert bench.read_traffic(1) is None  # the persistent form has no per-kernel summary
    f.write_text(f"- kernel_source_hash: {bench.source_hash(bench.TRAVERSE_SOURCES[2])}\n- traffic_bytes_per_ray: 123.0\n")
    assert bench.read_traffic(2) == 123.0

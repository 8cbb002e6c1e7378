"""The bench's multi-rank timing reduction on CPU: world size 2 over gloo
(the GPU runs use NCCL; each rank times its own replica and the slowest
rank's time is reported)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        q.put((rank, bench.max_over_ranks(1.5 + rank, "cpu"), bench.max_over_ranks(7.0 - rank, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2.5, 7.0), (1, 2.5, 7.0)]


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def _run_bench(env_extra, *args):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], env=env, cwd=root,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_rank_zero_only():
    """The reference arm (the CPU oracle, timed) prints one line on rank 0 and
    nothing on the other ranks, which exit 0 without work."""
    args = ("--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "3")
    assert _run_bench({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, *args) == []
    lines = _run_bench({"RANK": "0", "LOCAL_RANK": "0", "WORLD_SIZE": "1"}, *args)
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0

"""Multi-rank host logic on CPU with the gloo backend, world size 2.

The solves shard across GPUs with no exchange (one independent replica per
rank), so what crosses ranks is the bench's whole-job aggregation: the
slowest rank's step time (max over ranks) and every rank's bytes.  Checked
here with two gloo ranks, plus the reference arm under torchrun (rank 0 alone
runs and prints one JSON line, the other rank exits 0 without work).  No GPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BYTES = 1_000_000


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, val = bench.aggregate_ranks(1.0 + rank, BYTES, world, dist, "cpu")
    q.put((rank, ms, val))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_the_slowest_rank_and_all_bytes():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, val in res:
        assert ms == 2.0                      # rank 1's 2 ms, on both ranks
        assert val == pytest.approx(2 * BYTES / 2e-3 / 1e9, rel=1e-12)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, val = bench.aggregate_ranks(1.5, BYTES, 1)
    assert ms == 1.5
    assert val == pytest.approx(BYTES / 1.5e-3 / 1e9, rel=1e-12)


def test_reference_arm_two_ranks_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1                    # rank 0 alone prints
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0

"""The bench's multi-rank path on the host (gloo, world size 2): the job's
time is the slowest rank's (a MAX all-reduce), a sharded job's work and
root extents are sums over the ranks, and under torchrun the reference arm
runs on rank 0 alone, which prints the one JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    got = bench.max_over_ranks(1.5 + rank, ws)     # rank 1 is the slower one
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def _sum_rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    # a sharded DAG: each rank's flops, and each root's slices on this rank
    total = bench.sum_over_ranks(10.0 * (rank + 1), ws)
    lts = bench.sum_over_ranks([3 + rank, 2, 5 - rank], ws)
    out[rank] = (total, tuple(lts))
    dist.barrier()
    dist.destroy_process_group()


def test_sum_over_ranks_gloo_world_size_2():
    """The sharded bench sums the ranks' flops and each root's slices."""
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_sum_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert dict(out) == {0: (30.0, (7.0, 4.0, 9.0)), 1: (30.0, (7.0, 4.0, 9.0))}


def test_sum_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.sum_over_ranks(2.5, 1) == 2.5
    assert bench.sum_over_ranks([1, 2], 1) == [1.0, 2.0]


def test_max_over_ranks_gloo_world_size_2():
    ws = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_under_torchrun_world_size_2():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "tiny", "--steps", "1", "--warmup", "0", "--ref-seconds", "0.2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0

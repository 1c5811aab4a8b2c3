"""The N > 1 host path, on CPU with gloo ranks: every rank maps its own independent network,
and the only exchange (after the timed region) is the max of the ranks' times and the sum of
their node counts."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units, secs = bench.combine_ranks(100 * (rank + 1), 1.0 + 0.5 * rank, world)
        inst = bench.make_workload("tiny_plain_2x32x32", rank)
        out[rank] = (units, secs, float(np.sum(inst.gx)))
    finally:
        dist.destroy_process_group()


def test_combine_and_per_rank_networks():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r][0] == 300.0          # nodes of both ranks
        assert out[r][1] == 1.5            # the slowest rank's time
    assert out[0][2] != out[1][2]          # independent networks (own seeds)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(7, 0.25, 1) == (7.0, 0.25)


def test_reference_arm_under_torchrun_prints_one_line():
    """Rank 0 alone runs the reference arm (the oracle on the host cores) and prints one
    line; the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-sample", "32"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0

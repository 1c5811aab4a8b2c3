"""The N > 1 host paths, on CPU with gloo ranks.

Replicas: every rank maps its own independent network, and the only exchange (after the
timed region) is the max of the ranks' times and the sum of their node counts.

Column shards: every rank maps the same network over its share of the sketch columns and the
partial maps are summed by one all-reduce.  The ranks' partial maps come from the oracle's
same-seed Z split by columns; the reduced map must equal the single-rank map up to the
order of the sum."""
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


def test_column_shards_cover_the_sketch():
    sys.path.insert(0, ROOT)
    from paper_2607_05818_gb300.er import column_shard
    for k in (8, 36, 128, 256, 260):
        for world in (1, 2, 3, 4, 8):
            if k < 4 * world:
                continue
            cols = []
            for r in range(world):
                j0, kl = column_shard(k, world, r)
                assert kl % 4 == 0 and kl >= 4
                cols += list(range(j0, j0 + kl))
            assert cols == list(range(k))
    with pytest.raises(ValueError):
        column_shard(8, 3, 0)


def _shard_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from oracle import sketch as osk
    from paper_2607_05818_gb300 import instances as I
    from paper_2607_05818_gb300.er import column_shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst = I.random_small(np.random.default_rng(21), T=2, W=9, H=7, n_tsv=5, n_pads=2, open_frac=0.15)
        k, seed = 24, 99
        _, Z = osk.reff_jl_dense(inst, k, seed)            # the whole sketch's Z (oracle)
        j0, kl = column_shard(k, world, rank)
        part = torch.from_numpy(np.sum(Z[:, j0:j0 + kl] ** 2, axis=1))
        part[torch.from_numpy(np.all(Z == 0, axis=1))] = float("inf")  # floating nodes, as er_reff_map
        bench.reduce_partial_map(part, world)
        out[rank] = part.numpy()
    finally:
        dist.destroy_process_group()


def test_column_sharded_map_equals_single_rank():
    sys.path.insert(0, ROOT)
    from oracle import sketch as osk
    from paper_2607_05818_gb300 import instances as I
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_shard_main, args=(world, _free_port(), out), nprocs=world, join=True)
    inst = I.random_small(np.random.default_rng(21), T=2, W=9, H=7, n_tsv=5, n_pads=2, open_frac=0.15)
    R_full, _ = osk.reff_jl_dense(inst, 24, 99)
    fin = np.isfinite(R_full)
    assert (~fin).any()                                    # the instance has floating nodes
    for r in range(world):
        assert np.array_equal(np.isfinite(out[r]), fin)
        np.testing.assert_allclose(out[r][fin], R_full[fin], rtol=1e-14, atol=0)
    np.testing.assert_array_equal(out[0], out[1])          # every rank holds the same map

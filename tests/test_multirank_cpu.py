"""Multi-rank host logic on CPU with the gloo backend (world size 2): the
benchmark's whole-job aggregation (max time over ranks, sum of lattice
updates) and the round-robin sharding of independent cases.  The data path
itself has no collective: lattices are replicas."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    nodes = 1000 * (rank + 1)
    ms = 10.0 * (rank + 1)
    value, ms_max = bench.aggregate(nodes, 5, ms, dist)
    mine = bench.shard(range(11), rank, world)
    out[rank] = (value, ms_max, tuple(mine))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_and_shard_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    total_nodes = 1000 + 2000
    for r in range(world):
        value, ms_max, mine = out[r]
        assert ms_max == pytest.approx(20.0)
        assert value == pytest.approx(total_nodes * 5 / 0.020 / 1e6)
    assert sorted(out[0][2] + out[1][2]) == list(range(11))
    assert set(out[0][2]).isdisjoint(out[1][2])


def test_single_rank_aggregate():
    import bench
    value, ms = bench.aggregate(2048 * 1024, 100, 50.0)
    assert ms == 50.0 and value == pytest.approx(2048 * 1024 * 100 / 0.05 / 1e6)


def test_reference_arm_prints_on_rank_zero_only():
    """--impl reference: rank 0 times the oracle and prints one line; other ranks exit 0 silently."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--small", "--steps", "1",
           "--warmup", "1", "--ref-budget", "0.2"]
    for rank, expect_line in (("1", False), ("0", True)):
        env = dict(os.environ, RANK=rank, WORLD_SIZE="2")
        out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300, cwd=root)
        assert out.returncode == 0, out.stderr
        lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
        if expect_line:
            assert len(lines) == 1
            rec = json.loads(lines[0])
            assert rec["impl"] == "reference" and rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
        else:
            assert lines == []

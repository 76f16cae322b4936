"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

The product does not shard across GPUs in this build: N GPUs run N
independent replicas, and the only cross-rank steps are the barrier and the
max-over-ranks of the timed region.  These tests run that logic with two
gloo ranks and check the reference arm's rank rule (rank 0 alone works and
prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [12.0, 15.5][rank]                     # rank 1 is the slower replica
    ms = bench.replica_max(ms_local, world, "cpu")
    dist.barrier()
    value = bench.replica_value(world, 20, ms)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "value": value}, f)
    dist.destroy_process_group()


def test_replica_max_and_value_two_gloo_ranks(tmp_path):
    port = free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"r{i}.json")) for i in range(2)]
    assert r[0] == r[1]                                # every rank sees the slowest rank's time
    assert r[0]["ms"] == 15.5
    assert r[0]["value"] == pytest.approx(2 * 20 / 15.5e-3)


def test_replica_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(3.25, 1, "cpu") == 3.25
    assert bench.replica_value(1, 10, 100.0) == pytest.approx(100.0)


def test_reference_arm_other_ranks_exit_silently():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""

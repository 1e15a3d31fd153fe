"""The benchmark's multi-rank path on the CPU: two gloo ranks.  Replicas
train with different seeds, the job time is the slowest rank's, and only rank
0 prints; `--impl reference` on rank 1 exits without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": ms, "seed": bench.replica_seed(rank), "env": list(bench.dist_env())}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_max_and_use_distinct_seeds(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    r = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    assert r[0]["ms"] == r[1]["ms"] == 15.0
    assert r[0]["seed"] != r[1]["seed"]
    assert r[0]["env"][:2] == [0, 2] and r[1]["env"][:2] == [1, 2]
    del torch


def test_reference_arm_on_a_non_zero_rank_exits_silently():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0 and p.stdout.strip() == ""

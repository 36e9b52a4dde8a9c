"""Host logic of a multi-GPU bench run, on CPU: two gloo ranks, no GPU.

A run on N GPUs is N independent replicas (frames are independent units, no data-path
collective): each rank times its own frame, the ranks meet at barriers, the slowest
rank's times are taken by an all-reduce MAX, and the whole-job rate counts every rank's
pixels.  The reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w, lr = bench._dist()
    assert (r, w, lr) == (rank, world, rank)
    # per-rank times (ms): the job takes the slowest rank, element by element
    mine = [10.0 + rank, 5.0 - rank, 3.0 * (rank + 1)]
    dist.barrier()
    got = bench._max_over_ranks(dist, mine, "cpu")
    seed = bench._frame_spec(rank).seed
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"max": got, "seed": seed}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["max"] == [11.0, 5.0, 6.0]
    # each rank times its own frame
    assert res[0]["seed"] != res[1]["seed"]


def test_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    px = 2048 * 4096
    one = bench._job_rate(1, px, 100, 84.0)
    assert one == pytest.approx(px * 100 / 0.084 / 1e6)
    # weak scaling: N ranks with the same per-rank time give N times the rate
    assert bench._job_rate(4, px, 100, 84.0) == pytest.approx(4 * one)
    # the slowest rank sets the time
    assert bench._job_rate(2, px, 100, 168.0) == pytest.approx(one)


def test_reference_arm_only_on_rank0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""

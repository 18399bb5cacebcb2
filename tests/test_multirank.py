"""The replicas-only multi-GPU path, on CPU: two `gloo` ranks run the bench's
barrier, max-over-ranks timing and whole-job aggregation, and the reference arm
does no work on ranks other than 0.  (No GPU: the per-rank product is the
single-GPU path, covered by the GPU tests.)"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = [3.0, 7.5][rank]  # the second replica is slower
        ms_max = bench.max_over_ranks(ms, world)
        rate = bench.job_rate(1000.0, ms_max, world)
        bench.barrier(world)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms_max": ms_max, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_replica(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:
        assert g["ms_max"] == 7.5  # both ranks see the slowest time
        assert g["rate"] == pytest.approx(2 * 1000.0 / 7.5e-3)  # units of all ranks / max time


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, 1) == 4.0
    assert bench.job_rate(500.0, 2.0, 1) == pytest.approx(250000.0)


def test_reference_arm_does_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""  # rank 0 alone runs and prints

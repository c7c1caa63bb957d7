"""The N > 1 host path of the benchmark (replicas: one process per GPU, no data exchange)
with world size 2 on the gloo backend: max-over-ranks timing, whole-job throughput, and the
reference arm running on rank 0 only."""
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
    t = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    out[rank] = (t, bench.job_geris(1_000_000_000, world, t))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, g = res[r]
        assert t == 15.0  # every rank reports the slowest replica's time
        assert g == pytest.approx(2 * 1e9 / 15e-3 / 1e9)  # ERIs of both replicas / that time


def test_single_process_has_no_collective():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_geris(2_000_000_000, 1, 1000.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""  # rank 1 does no work and prints nothing

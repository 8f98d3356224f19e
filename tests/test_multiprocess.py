"""The N-replica path of bench.py on CPU: two gloo ranks, no GPU.

Frames are independent (one fusion per time step, no state carried between frames), so N
GPUs run N replicas with no data-path collective; the only collectives are the timing
barrier and the max-over-ranks reduction, exercised here with the gloo backend.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = 100.0 + 50.0 * rank                       # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, world)
    rate = bench.job_rate(1000.0, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{slowest} {rate}\n")


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    vals = [open(tmp_path / f"r{r}.txt").read().split() for r in range(2)]
    for slowest, rate in vals:
        assert float(slowest) == 150.0
        # 2 ranks x 1000 units in 0.150 s
        assert abs(float(rate) - 2000.0 / 0.150) < 1e-6


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(10.0, 1, 1000.0) == 10.0


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""

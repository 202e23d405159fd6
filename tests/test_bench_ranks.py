"""The multi-GPU (replicas) arithmetic of bench.py on CPU: two gloo ranks.

Each rank runs its own replica; the job time is the slowest rank's time (an
all-reduce MAX) and the whole-job throughput counts every rank's iterations.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dt = 1.0 + 0.5 * rank                      # rank 1 is the slow replica
    dt_max = bench.max_over_ranks(dt, dist, torch.device("cpu"))
    out[rank] = (dt_max, bench.job_throughput(20, world, dt_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_job_throughput():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        dt_max, thr = out[r]
        assert dt_max == 1.5
        assert thr == pytest.approx(world * 20 / 1.5)


def test_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.job_throughput(10, 1, 2.0) == 5.0


def test_reference_arm_contract():
    """bench.py --impl reference on the small workload: one JSON line whose steps
    were all timed (ms_per_step x steps is the time that ran), on the host cores
    it reports, with the reference-arm keys the contract asks for."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "3", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 3
    assert line["unit"] == "iter/s" and line["higher_is_better"] is True
    assert line["value"] == pytest.approx(1e3 / line["ms_per_step"], rel=1e-9)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["final_state"]["it"] == 6   # warm-up and timed steps, every one a full iteration

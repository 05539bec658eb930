"""The multi-rank logic of bench.py on CPU: two gloo ranks (replicas only, no data-path
collective) reduce their timings to the maximum, and the whole-job rate counts the steps
of every rank over the slowest one; the reference arm prints on rank 0 only."""
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    # rank r "took" 1 + r seconds for its timed steps and 5 - r seconds end to end
    dev, e2e = bench.reduce_max_over_ranks([1.0 + rank, 5.0 - rank], world)
    with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as f:
        f.write("%r %r %r\n" % (dev, e2e, bench.whole_job_rate(world, 10, dev)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_maximum(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        dev, e2e, rate = open(tmp_path / ("r%d.txt" % r)).read().split()
        assert float(dev) == 2.0 and float(e2e) == 5.0
        assert float(rate) == 2 * 10 / 2.0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks([0.5, 0.25], 1) == [0.5, 0.25]
    assert bench.whole_job_rate(1, 10, 0.5) == 20.0


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--L", "129", "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--L", "129",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["metric"] == "RK steps/s"


def test_energy_threshold_of_the_aging_workload():
    """Sec. 4.3: the generic E_th formula gives -sqrt(2(p-1)/p) for pure models f = q^p/2
    (p = 3: -sqrt(4/3)) and -1 for the pure 2-spin model."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    for p in (2, 3, 4, 5):
        assert abs(bench.energy_threshold({p: 0.5}) + np.sqrt(2.0 * (p - 1) / p)) < 1e-15
    assert abs(bench.energy_threshold({2: 0.5}) + 1.0) < 1e-15

"""The multi-rank path of bench.py on CPU: gloo ranks (world size 2) agree on the slowest rank's
time, the whole-job rate counts every rank's units, every rank solves its own seeded instance,
and the oracle arm runs on rank 0 only."""

import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, world, "cpu")
        rate = bench.whole_job_rate(3, world, ms)
        c = bench.WORKLOADS["4x4"][0](instance=rank)
        fam = bench.WORKLOADS["batch"][0](instance=rank)
        np.savez(os.path.join(out_dir, "r%d.npz" % rank), ms=ms, rate=rate, t=c["t"],
                 U=np.array([f["U"][0] for f in fam[:16]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    r = [np.load(tmp_path / ("r%d.npz" % k)) for k in range(world)]
    assert float(r[0]["ms"]) == float(r[1]["ms"]) == 150.0
    assert abs(float(r[0]["rate"]) - 2 * 3 / 0.150) < 1e-9
    assert not np.array_equal(r[0]["t"], r[1]["t"])      # the seeded t' signs differ per rank
    assert not np.array_equal(r[0]["U"], r[1]["U"])      # and so do the batched families


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_rate(4, 1, 2000.0) == 2.0


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""

"""The multi-rank path of bench.py on CPU: world-size-2 gloo ranks on 127.0.0.1. Ranks are
independent replicas (each its own seeded bed, no collective on the data path); the only
collective is the max over ranks of the timed region, and the job's throughput counts every
rank's parcels over that slowest time. The reference arm runs on rank 0 only."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank                 # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms_local, dist, "cpu")
        bed = bench.make_workload("plain_2k", rank, 0)
        out[rank] = (ms_max, bench.job_throughput(bed.n, world, 100, ms_max), float(bed.x.sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_own_beds():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (m0, v0, x0), (m1, v1, x1) = out[0], out[1]
    assert m0 == m1 == 15.0                          # both see the slowest rank's time
    assert v0 == v1 == 2000 * world * 100 / 15e-3    # all parcels of both ranks over that time
    assert x0 != x1                                  # each rank steps its own seeded replica


def test_single_rank_is_its_own_maximum():
    assert bench.max_over_ranks(3.5) == 3.5
    assert np.isclose(bench.job_throughput(1000, 1, 10, 2.0), 5e6)


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    bench.reference_arm(bench.parse())
    assert capsys.readouterr().out == ""

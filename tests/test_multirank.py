"""The multi-rank path of the benchmark on CPU with gloo, world size 2 (replicas: every rank solves
its own box, no collective on the data path): each rank gets its own seeded box, the job time is
the slowest rank's and the job's interactions are the sum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        pos, mass, eps, theta = bench.workload("plummer4096", rank)
        ms, inter = bench.job_totals(10.0 + rank, 1000.0 * (rank + 1), world, "cpu")
        out[rank] = (float(pos[0, 0]), float(pos[1, 7]), ms, inter, eps, theta)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_get_distinct_boxes():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork: earlier tests may have started OpenMP threads
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    (x0, y0, ms0, in0, e0, t0), (x1, y1, ms1, in1, e1, t1) = res[0], res[1]
    assert (x0, y0) != (x1, y1)  # independent seeded boxes
    assert ms0 == ms1 == 11.0  # the slowest rank's time
    assert in0 == in1 == 3000.0  # interactions of both ranks
    assert (e0, t0) == (e1, t1)


def test_single_rank_totals_are_local():
    import bench

    assert bench.job_totals(5.0, 7.0, 1, "cpu") == (5.0, 7.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench

    class A:
        workload, n, cpu_sample, steps, warmup, gpus = "plummer4096", None, None, 1, 0, 2

    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""

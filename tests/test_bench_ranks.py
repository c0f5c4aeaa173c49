"""The replicas path of bench.py on CPU: two gloo ranks, max-over-ranks timing, whole-job value,
and the reference arm doing no work on ranks other than 0."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms, value = bench.job_time_and_value(10.0 + 5.0 * rank, 1000, ws, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_points():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms, value = res[r]
        assert ms == 15.0                        # the slower rank's time on every rank
        assert value == pytest.approx(2 * 1000 / 0.015)


def test_single_rank_value():
    import bench
    assert bench.job_time_and_value(20.0, 500, 1) == (20.0, pytest.approx(500 / 0.02))


def test_reference_arm_other_ranks_exit_without_work(capsys):
    import argparse

    import bench
    args = argparse.Namespace(workload="sphere4k", digits=0, steps=1, warmup=0)
    assert bench.run_reference(args, ws=2, rank=1) == 0
    assert capsys.readouterr().out == ""

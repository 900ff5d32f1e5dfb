"""The multi-GPU form of bench.py is N independent replicas (weak scaling, no data-path
collective): each rank times its own steps, the job's time is the slowest rank's, and the
value is the units all ranks processed over that time.  The host side of that is checked
here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 10.0 + 5.0 * rank                   # rank 1 is the slower one
    t = bench.max_over_ranks(t_local, dist, torch.device("cpu"))
    out[rank] = (t, bench.whole_job_rate(1000.0, 4, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, v = res[0]
    assert t == 15.0
    assert v == pytest.approx(1000.0 * 4 * 2 / 0.015)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.whole_job_rate(10.0, 2, 1, 4.0) == pytest.approx(5000.0)


def test_reference_arm_other_ranks_exit_without_work(capsys):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(None, 1, 2) == 0
    assert capsys.readouterr().out == ""

"""The N > 1 host logic of the benchmark on CPU ranks (gloo, world size 2): replicas
only, so the one exchange is the max over ranks of the step time; the whole-job value
counts every rank's bodies over the slowest rank's time; the reference arm runs on
rank 0 alone."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = [3.5, 7.25][rank]                  # rank 1 is the slower one
        dist.barrier()
        t_max = bench.max_over_ranks(t, world, "cpu")
        out[rank] = (t_max, bench.whole_job_value(1000, world, t_max))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_two_ranks():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t_max, value = res[rank]
        assert t_max == 7.25                   # every rank sees the slowest time
        assert value == pytest.approx(2 * 1000 / 7.25e-3)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.max_over_ranks(4.0, 1) == 4.0
    assert bench.whole_job_value(500, 1, 2.0) == pytest.approx(250000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
        args = bench.parse()
    finally:
        sys.argv = sys_argv
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""

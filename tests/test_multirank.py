"""CPU test of the multi-GPU bench path with world_size 2 over gloo: independent pairs per rank
(weak scaling, no data-path collective), max-over-ranks timing, whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        t_step, t_e2e = bench.reduce_max_over_ranks([1.0 + rank, 3.0 - rank])
        out[rank] = (t_step, t_e2e, bench.whole_job_rate(1, world, t_step))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_time():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t_step, t_e2e, rate = out[r]
        assert t_step == 2.0 and t_e2e == 3.0          # max over ranks on every rank
        assert rate == pytest.approx(1.0)              # 2 pairs over the slowest rank's 2 s


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.whole_job_rate(1, 1, 0.5) == 2.0

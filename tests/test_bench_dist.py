"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each an
independent replica, combine their timings the way the benchmark does
(max over ranks for time, sum over ranks for units)."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, lr = bench.dist_env()
    assert (w, r, lr) == (world, rank, rank)
    d = bench.dist_init(w, "gloo")
    seconds = [1.5, 2.5][rank]
    units = [100.0, 300.0][rank]
    mx = bench.reduce_max(d, seconds)
    tot = bench.reduce_sum(d, units)
    out[rank] = (mx, tot, bench.whole_job_rate(tot, mx))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == (2.5, 400.0, 160.0)


def test_single_rank_identity():
    import bench
    assert bench.reduce_max(None, 3.0) == 3.0
    assert bench.reduce_sum(None, 4.0) == 4.0
    assert bench.whole_job_rate(10.0, 2.0) == 5.0

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


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, capture_output=True, text=True,
                       env=env, cwd=root, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    # the reference arm (the oracle on this host's cores) prints one line with
    # the contract's keys, on the same metric as our arm
    out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3", "--workload", "er_n1000_m5000_k3",
                      "--reference-roots", "50"])
    assert len(out) == 1
    d = out[0]
    import bench
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "er_n1000_m5000_k3"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3", "--workload", "er_n1000_m5000_k3",
                      "--reference-roots", "10"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out == []


def test_reference_arm_times_the_whole_workload_by_default():
    # without --reference-roots every ESU root is counted in each step: the
    # same config as our arm, not a sample of it
    out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3", "--workload", "er_n1000_m5000_k3"])
    assert len(out) == 1
    d = out[0]
    assert d["cpu_baseline"]["sample"].startswith("the whole workload, all 1000 ESU roots (44842 subgraphs")

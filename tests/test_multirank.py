"""The multi-GPU path of bench.py (independent replicas, one per rank) on
CPU: two gloo ranks agree on the slowest rank's time, the whole-job rate
counts both ranks' steps, and each rank's replica has its own seed. Runs
without a GPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        local_ms = [120.0, 175.5][rank]
        ms_max = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ms_max, bench.whole_job_rate(world, 10, ms_max), bench.replica_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 175.5
    assert res[0][1] == res[1][1] == pytest.approx(2 * 10 / 0.1755)
    assert res[0][2] != res[1][2]


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(42.0, None, "cpu") == 42.0
    assert bench.whole_job_rate(1, 10, 500.0) == pytest.approx(20.0)
    assert bench.replica_seed(0) == 2106


def test_cpu_legs_share_one_bounded_sample():
    # the bench arm's cpu_baseline and the reference arm take the same sample
    assert bench.sample_planes(20, 5) == 16
    assert bench.sample_planes(1, 3) == 16
    for k, w in [(50, 5), (200, 10), (26, 0)]:
        n = bench.sample_planes(k, w)
        assert n % 2 == 0 and 8 <= n < 16
        assert n * (k + w) <= 16 * 25 or n == 8

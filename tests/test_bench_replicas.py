"""The benchmark's multi-GPU path is replicas only (the hot path does not shard:
no data-path collective).  Its host logic -- the slowest replica's time sets
the whole job's, the value counts every replica's particles, only rank 0
reports, the reference arm runs on rank 0 alone -- is checked here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (r + 1) ms for the step loop and 10 (r + 1) ms end to end
        got = bench.max_over_ranks(rank + 1.0, 10.0 * (rank + 1))
        out[rank] = got
    finally:
        td.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == [2.0, 20.0]


def test_max_over_ranks_without_a_group_is_the_identity():
    assert bench.max_over_ranks(3.0, 4.5) == [3.0, 4.5]


def test_whole_job_rate_counts_every_replica_over_the_slowest_time():
    # 1e6 particles per replica, 2 replicas, 10 steps, slowest replica 20 ms
    assert bench.whole_job_rate(1_000_000, 2, 10, 20.0) == pytest.approx(1e9)
    assert bench.whole_job_rate(1_000_000, 1, 10, 20.0) == pytest.approx(5e8)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        workload, steps, warmup, threads = "weibel_512", 1, 3, 256
    assert bench.run_reference(A(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""

"""The N > 1 path of bench.py on the CPU: world-size-2 gloo process groups.

bench.py runs one replica of the workload per GPU (the path shards with no
exchange step), takes the job's time as the slowest rank's, and reports the
whole job's throughput.  These tests run that host logic with the gloo backend
on 127.0.0.1; the GPU runs use the same functions over NCCL."""
import socket
import sys

import pytest

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(dist, times[rank])
        rate = bench.job_rate(world, 1000.0, 5, slowest)
        dist.barrier()
        q.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time_gloo():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    times = [0.75, 1.25]   # seconds on rank 0 and rank 1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    # every rank sees the slowest time, and the job's rate counts both replicas
    assert got == [(0, 1.25, 2 * 1000.0 * 5 / 1.25), (1, 1.25, 2 * 1000.0 * 5 / 1.25)]


def test_single_process_is_its_own_maximum():
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.job_rate(1, 6.0e8, 10, 0.5) == pytest.approx(1.2e10)


def test_job_rate_is_weak_scaling():
    # fixed work per rank: N ranks in the same time do N times the work
    one = bench.job_rate(1, 6.0e8, 10, 0.6)
    assert bench.job_rate(4, 6.0e8, 10, 0.6) == pytest.approx(4 * one)


def test_other_ranks_of_the_reference_arm_do_no_work(monkeypatch, capsys):
    # under torchrun only rank 0 times the oracle and prints the line
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    args = bench.parse()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""

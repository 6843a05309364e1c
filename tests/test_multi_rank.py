"""The several-GPU path of the benchmark is independent replicas: each rank
generates its own instance (seed + rank), the ranks meet at a barrier around
the timed region, and the job's time is the slowest rank's. The host side of
that is checked here with world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_max = bench.max_over_ranks(local_ms[rank], "cpu", world)
        dist.barrier()
        out.put((rank, ms_max, bench.replica_seed(3, rank),
                 bench.job_throughput(1000.0, 5, world, ms_max)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, local_ms = 2, [3.0, 5.0]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, local_ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5.0, 5.0]                 # both ranks see the max
    assert [r[2] for r in res] == [3, 4]                     # distinct instances
    # 1000 units per rank per step, 5 steps, 2 ranks, 5 ms -> 2e6 units/s
    assert all(abs(r[3] - 1000.0 * 5 * 2 / 0.005) < 1e-6 for r in res)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5, "cpu", 1) == 7.5
    assert bench.job_throughput(10.0, 2, 1, 1000.0) == 20.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        workload = "ba_n100k_m4"
        steps, warmup = 1, 0
    assert bench.run_reference(A(), rank=1, world=2) == 0
    assert capsys.readouterr().out == ""

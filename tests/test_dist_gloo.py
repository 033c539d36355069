"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2) time
independent replicas; the job is timed by the slowest rank and the throughput
counts every rank's cells."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    elapsed = [12.5, 20.0][rank]  # rank 1 is the slow one
    m = bench.max_over_ranks(elapsed, world)
    out[rank] = (m, bench.job_mlups(world, 1000, 10, m))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        m, mlups = out[r]
        assert m == 20.0
        assert mlups == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_reference_arm_other_ranks_do_no_work():
    import argparse

    import bench
    args = argparse.Namespace(steps=3, warmup=3, workload="d2q9_64_fp64", gpus=2)
    assert bench.run_reference(args, world=2, rank=1) == 0

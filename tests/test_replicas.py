"""The N > 1 bookkeeping of bench.py on CPU ranks (gloo, world size 2): one
process per rank, each with its own lattice and no data-path collective;
only the timings meet (barrier, maximum over ranks), and the whole-job value
is every rank's cell updates over the slowest rank's time.  The reference
arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        local_seconds = [0.5, 2.0][rank]          # the second rank is slower
        dist.barrier()
        slowest = bench.max_over_ranks(local_seconds, dist)
        value = bench.whole_job_mlups(world, 1_000_000, slowest)
        # the reference arm does its work on rank 0 only
        args = type("A", (), {"steps": 1, "warmup": 3, "n": 8})()
        ran = rank == 0
        if rank != 0:
            assert bench.run_reference(args, rank, world) is None
        q.put((rank, slowest, value, ran))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value, _ in got:
        assert slowest == 2.0                          # max over ranks, on every rank
        assert value == pytest.approx(2 * 1_000_000 / 2.0 / 1e6)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, None) == 1.25
    assert bench.whole_job_mlups(1, 2_097_152, 0.1) == pytest.approx(20.97152)

"""Multi-rank timing of the replica benchmark on CPU (gloo, world size 2).

The solve has no exchange step on one gauge field, so N GPUs run N independent
replicas; the only cross-rank operations are the barrier and the MAX of the
per-rank times.  These tests run that host logic as two gloo processes.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 7.5 * rank)        # rank r took 10 + 7.5 r ms
        dist.barrier()
        out[rank] = (ms, bench.job_rate(world, 5, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    slow = 10.0 + 7.5 * (world - 1)
    for r in range(world):
        ms, rate = out[r]
        assert ms == slow                                   # every rank sees the slowest replica
        assert rate == pytest.approx(world * 5 / (slow / 1e3))


def test_single_process_is_identity():
    import bench
    assert not (dist.is_available() and dist.is_initialized())
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_rate(1, 5, 1000.0) == pytest.approx(5.0)


def _ref_rank_main(rank, world, port, out):
    # the reference arm: rank 0 alone runs the oracle; other ranks return without work
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    class Args:
        steps = 1

    called = []
    bench.make_inputs = lambda w: called.append(1) or (_ for _ in ()).throw(RuntimeError("rank 0 work"))
    try:
        bench.run_reference(Args(), None)
        out[rank] = "returned"
    except RuntimeError:
        out[rank] = "worked"


def test_reference_arm_rank0_only():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_ref_rank_main, args=(2, 0, out), nprocs=2, join=True, start_method="spawn")
    assert out[1] == "returned"
    assert out[0] == "worked"

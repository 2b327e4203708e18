"""The multi-GPU path is replicas only: each rank solves its own parameter
vectors, and the only cross-rank step is the timing reduction (the slowest
rank's time).  This checks that host logic with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        per_rank_ms = [120.0, 80.0][rank]
        ms = bench.max_over_ranks(per_rank_ms)
        seeds = [bench.replica_request(rank, i) for i in range(16)]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out[rank] = (ms, bench.whole_job_rate(16, world, ms), gathered)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_disjoint_parameters():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, rate, gathered = out[r]
        assert ms == 120.0  # both ranks report the slowest rank's time
        assert rate == pytest.approx(2 * 16 / 0.120)  # whole-job units per second
        assert not set(gathered[0]) & set(gathered[1])  # no parameter solved twice


def test_single_rank_needs_no_process_group():
    assert not dist.is_initialized()
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.whole_job_rate(16, 1, 1000.0) == pytest.approx(16.0)

"""The multi-GPU form is N independent replicas (the method has no data-parallel exchange at these
sizes): the benchmark's whole-job figures are the slowest rank's time and all ranks' launches.
Two gloo ranks on the CPU (no GPU)."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, port: int, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        import bench
        times = [120.0, 155.5]
        launches = [1000, 1003]
        out[rank] = bench.replica_totals(times[rank], launches[rank], dist, None)
    finally:
        dist.destroy_process_group()


def test_replica_totals_take_the_slowest_rank_and_all_launches():
    port = _free_port()
    ctx = mp.get_context("spawn")  # no fork of a process that may hold threads (an OpenMP oracle build)
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (155.5, 2003)


def test_replica_totals_without_a_group_are_local():
    import bench
    assert bench.replica_totals(42.0, 7) == (42.0, 7)

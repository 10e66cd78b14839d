"""The replica logic of bench.py under torch.distributed on CPU (gloo,
world_size 2): environment parsing, barrier, the maximum over ranks and the
whole-job throughput from the slowest rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench.dist_env()
        dist.barrier()
        # rank r "took" 10 (r + 1) ms for 100 steps of 7 units
        t_max = bench.max_over_ranks(torch, 10.0 * (rank + 1), got_ws)
        value = bench.replica_value(got_ws, 100 * 7, t_max)
        q.put((rank, got_ws, got_rank, got_local, t_max, value))
    finally:
        dist.destroy_process_group()


def test_replicas_report_the_slowest_rank():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, got_ws, got_rank, got_local, t_max, value in out:
        assert (got_ws, got_rank, got_local) == (2, rank, rank)
        assert t_max == 20.0
        assert value == pytest.approx(2 * 700 / 0.020)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(torch, 3.5, 1) == 3.5
    assert bench.replica_value(1, 10, 1000.0) == pytest.approx(10.0)

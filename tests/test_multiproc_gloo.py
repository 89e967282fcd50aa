"""The replicated multi-GPU path of the benchmark, on CPU with two gloo ranks.

Tracks are independent, so N GPUs run N replicas with no data-path collective;
the only collective is the max over ranks of the timed region, and the
whole-job value is the units of all ranks over that time.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.0, 20.0][rank]
    ms_max = bench.reduce_max(ms, world, device="cpu")
    val = bench.aggregate(1000.0, world, ms_max)
    dist.barrier()
    q.put((rank, ms_max, val))
    dist.destroy_process_group()


def test_replicas_reduce_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]
    assert res[0][2] == pytest.approx(2 * 1000.0 / 0.020)


def test_single_rank_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.aggregate(10.0, 1, 1000.0) == pytest.approx(10.0)

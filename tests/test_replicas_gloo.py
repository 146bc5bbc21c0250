"""Host logic of the multi-GPU bench path (independent replicas, one image per rank) on
two CPU ranks with the gloo backend: the slowest rank's time decides, and the whole-job
throughput counts every rank's pixels."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slower replica
        m = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (m, bench.replica_throughput(m, world, 512, 768, 10))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    m, v = res[0]
    assert m == 150.0
    assert v == pytest.approx(2 * 512 * 768 * 10 / 0.150 / 1e6)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(1000.0, 1, 10, 10, 5) == pytest.approx(5e-4)

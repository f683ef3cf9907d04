"""The bench's N-GPU mode runs independent replicas (the step has no exchange on one
GPU): its whole-job rate takes the slowest rank's time and every rank's particles.
Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ms, value = bench.replica_rate(10.0 + 5.0 * rank, 1000, 4, dist)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
    for r in range(2):
        ms, value = out[r]
        assert ms == 15.0                       # the slower rank
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)


def test_replica_rate_single_process():
    import bench

    ms, value = bench.replica_rate(8.0, 500, 2, None)
    assert ms == 8.0 and value == pytest.approx(500 * 2 / 0.008)

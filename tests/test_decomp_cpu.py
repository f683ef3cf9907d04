"""The cycle sharded by x-slabs over 2 and 3 CPU ranks (gloo), each rank running the
oracle on its slab with halo exchange, current fold and particle migration
(tests/decomp_oracle.py), gives the single-box oracle's fields and particles: the
layout the multi-GPU path would take, checked without GPUs."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2609_16575_gb300 import workloads as W

STEPS = 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case():
    wl = W.thermal((24, 6, 6), 0.2, 2, 0.3, seed=121)
    n, d, dt = wl.n, wl.d, wl.dt
    F = oracle.empty_fields(n)
    # a standing field so that E and B are non-zero everywhere from the start
    kk, jj, ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    F[1] = 0.05 * np.sin(2 * np.pi * ii / n[0]) * (1 + 0.2 * np.cos(2 * np.pi * kk / n[2]))
    F[5] = 0.03 * np.cos(2 * np.pi * (ii + 0.5) / n[0])
    return n, d, dt, F, wl.species[0].P


def _rank(rank, world, port, out):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch.distributed as dist

    from decomp_oracle import Slab

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, d, dt, F, P = _case()
    slab = Slab(n, d, dt, F, P, -1.0, 1.0, rank, world)
    for _ in range(STEPS):
        slab.step()
    Fs, ids, Ps = slab.result()
    out[rank] = (Fs, ids, Ps, slab.migrated, slab.folded)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_decomposition_equals_one_box(world):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    n, d, dt, F, P = _case()
    sp = [oracle.Species(-1.0, 1.0, P)]
    oracle.run(n, d, dt, F, sp, STEPS)
    Fd = np.concatenate([out[r][0] for r in range(world)], axis=3)
    scale = np.abs(F).max()
    assert np.abs(Fd - F).max() <= 1e-13 * scale, np.abs(Fd - F).max() / scale
    ids = np.concatenate([out[r][1] for r in range(world)])
    Pd = np.concatenate([out[r][2] for r in range(world)], axis=1)
    assert np.array_equal(np.sort(ids), np.arange(P.shape[1]))     # every particle once
    Q = sp[0].P
    Pd = Pd[:, np.argsort(ids)]
    dx = Pd[0:3] - Q[0:3]
    for k in range(3):
        dx[k] = (dx[k] + n[k] / 2) % n[k] - n[k] / 2
    assert np.abs(dx).max() <= 1e-12
    assert np.abs(Pd[3:7] - Q[3:7]).max() <= 1e-13 * np.abs(Q[3:6]).max()
    assert sum(out[r][3] for r in range(world)) > 0      # particles crossed slab faces
    assert sum(out[r][4] for r in range(world)) > 0      # current was folded

"""The N>1 path of the benchmark on CPU ranks (gloo, world size 2): each rank runs its own
coupling draw (replicas), the slowest rank's time sets the throughput, nothing else is
exchanged."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    from paper_2002_05725_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(100.0 + 50.0 * rank, "cpu", world)
        v = bench.curves_per_hour(world, 16, 2, t)
        J = inputs.couplings(12, seed=0, realization=rank)   # each rank: its own coupling draw
        out[rank] = (t, v, float(J[0]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    (t0, v0, j0), (t1, v1, j1) = out[0], out[1]
    assert t0 == t1 == 150.0                                  # max over ranks
    assert v0 == v1 == pytest.approx(2 * 16 * 2 * 3600.0 / 0.150)
    assert j0 != j1                                           # independent replicas


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, "cpu", 1) == 12.5
    assert np.isclose(bench.curves_per_hour(1, 16, 2, 10000.0), 16 * 2 * 0.36 * 1000)

"""The multi-rank (independent replica) logic of bench.py on CPU with the gloo
backend, world size 2: whole-job time is the slowest rank's, iterations add up,
and each rank draws its own configurations."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    T, n = bench.reduce_over_ranks(dist, 1.5 + rank, 10 * (rank + 1), device="cpu")
    U = bench.configs((4, 4, 4, 4), rank)
    out[rank] = (T, n, float(np.abs(U[0]).sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5  # max over ranks
    assert res[0][1] == res[1][1] == 30.0  # sum over ranks
    assert res[0][2] != res[1][2]  # independent replicas draw different fields

"""Multi-replica host logic of bench.py on CPU: two gloo ranks on 127.0.0.1 agree on
the max-over-ranks time, pass the barrier, and draw distinct per-rank workloads."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import workloads as W
    w, r, local = bench.dist_setup(world, "gloo")
    assert (w, r) == (world, rank)
    m = bench.reduce_max(10.0 * (rank + 1), w, None)
    bench.barrier(w)
    reqs = W.served_requests(count=5, seed=5 + rank)
    out[rank] = (m, reqs[0]["arrival"], W.config_2d(N=63, nt=64, seed=2 + 1000 * rank).f[0, 0])
    dist.destroy_process_group()


def test_two_rank_gloo_coordination():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a threaded process
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0          # max over ranks
    assert res[0][1] != res[1][1]                  # independent request streams
    assert res[0][2] != res[1][2]                  # independent problem instances (weak scaling)

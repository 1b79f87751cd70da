"""Multi-rank logic of bench.py on CPU (gloo, world size 2): replicas get distinct seeds, the
timing is the maximum over ranks, and the aggregate rate counts every rank's site updates."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    seed = bench.replica_seed(7, r)
    elapsed = 1.0 + r  # rank 1 is the slow one
    bench.barrier(w)
    t = bench.max_over_ranks(elapsed, w)
    out[rank] = (seed, t, w)
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (s0, t0, w0), (s1, t1, w1) = out[0], out[1]
    assert w0 == w1 == 2
    assert s0 != s1 and s0 == bench.replica_seed(7, 0)
    assert t0 == t1 == 2.0
    units = 1000
    assert world * units / max(t0, t1) == pytest.approx(1000.0)


def test_single_rank_defaults():
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5

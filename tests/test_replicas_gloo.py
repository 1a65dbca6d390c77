"""The multi-GPU form of the benchmark is independent replicas (one column per rank,
no collective in the data path).  Its host logic runs here as two gloo ranks on the
CPU: each rank builds a different replica (seed and RNG column), and the whole-job
figures are the slowest rank's time and the units of all ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2202_03215_gb300 import workloads as w


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = bench.replica_params(w, rank, 1000)
    seconds = [2.0, 3.5][rank]
    units = [100, 250][rank]
    t, u = bench.aggregate(dist, torch, seconds, units, device="cpu")
    q.put((rank, p.seed, p.column, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    (r0, s0, c0, t0, u0), (r1, s1, c1, t1, u1) = got
    assert (s0, c0) != (s1, c1)               # independent replicas
    assert t0 == t1 == 3.5 and u0 == u1 == 350


def test_single_rank_is_the_identity():
    assert bench.aggregate(None, torch, 1.25, 7) == (1.25, 7)

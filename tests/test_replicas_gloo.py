"""The multi-GPU form is replicas (independent searches, one per rank, no
data exchanged): the bench's cross-rank combination takes the slowest rank's
times and the sum of the configurations scored.  Checked with two gloo ranks
on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, e, n = bench.combine_ranks(dist, 1.0 + rank, 2.0 - rank, 1000 * (rank + 1), "cpu")
    q.put((rank, t, e, n))
    dist.destroy_process_group()


def test_two_rank_combination():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, e, n in got:
        assert (t, e, n) == (2.0, 2.0, 3000.0)


def test_single_process_passthrough():
    import bench
    assert bench.combine_ranks(None, 1.5, 2.5, 7, "cpu") == (1.5, 2.5, 7.0)

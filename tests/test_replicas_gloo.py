"""Replica path of bench.py on CPU: world_size-2 gloo ranks (no GPU).

The sector path does not shard across GPUs here (one GPU per box): N ranks
run N independent replicas, joined only by a barrier and by the
max-over-ranks timing reduction.  This checks that aggregation with two
gloo processes on 127.0.0.1."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist, r, ws = bench._dist()
    assert (r, ws) == (rank, world)
    bench._barrier(dist)
    # rank 0: 10 GB in 2 s; rank 1: 30 GB in 4 s -> 40 GB / 4 s = 10 GB/s
    nbytes = 10e9 if rank == 0 else 30e9
    secs = 2.0 if rank == 0 else 4.0
    iters = 100 if rank == 0 else 300
    v, it, tmax = bench.combine_ranks(dist, nbytes, iters, secs)
    q.put((rank, v, it, tmax))
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, v, it, tmax in out:
        assert tmax == pytest.approx(4.0)
        assert v == pytest.approx(10.0)
        assert it == pytest.approx(100.0)

"""World-size-2 CPU (gloo) test of the bench's cross-rank step: replicas are
independent, so ranks only combine their timed seconds (max) and their
evaluation counts (sum)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs, evals = bench.reduce_over_ranks(1.0 + rank, 100 * (rank + 1), dist, "cpu")
    out[rank] = (secs, evals)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 300.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(2.5, 42) == (2.5, 42.0)

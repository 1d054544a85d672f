"""The N > 1 host path of bench.py on CPU: two gloo ranks, barrier and max-over-ranks timing.

The benchmark runs the workload as replicas (no data exchange between GPUs): each rank
runs the whole workload, so the only collectives are the barrier and the timing reduction.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench

    d = bench.Dist()
    d.barrier()
    v = d.max(float(rank + 1) * 0.5)
    out[rank] = v
    d.close()


@pytest.mark.timeout(120)
def test_two_rank_barrier_and_max():
    ctx = mp.get_context("spawn")
    world = 2
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(100)
        assert all(p.exitcode == 0 for p in procs)
        assert dict(out) == {0: 1.0, 1: 1.0}

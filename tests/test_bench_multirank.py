"""Host logic of bench.py's multi-rank mode on CPU with world size 2 (gloo): each rank runs an
independent replica; the job time is the maximum over ranks and the value counts every rank's
updates."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 100.0 + 50.0 * rank  # rank 1 is slower
    slowest = bench.max_over_ranks(my_ms, "cpu")
    out[rank] = (slowest, bench.aggregate_mlups(world, 1000, 10, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_world2():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # 2 ranks x 1000 cells x 10 steps in 150 ms
    assert res[0][1] == pytest.approx(2 * 1000 * 10 / 0.150 / 1e6)

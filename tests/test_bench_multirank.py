"""The multi-rank aggregation of bench.py (replicas, max over ranks) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 if rank == 0 else 250.0          # rank 1 is the slow replica
    ms_max, value = bench.aggregate(ms, 1e6 * 4, world)
    out[rank] = (ms_max, value)
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        for r in range(2):
            ms_max, value = out[r]
            assert ms_max == 250.0
            assert value == pytest.approx(2 * 4.0 / 0.25)   # 2 ranks x 4 Mpoints / 0.25 s

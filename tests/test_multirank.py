"""The benchmark's N > 1 path runs one replica per rank; its whole-job
figure is the sum of all ranks' units over the slowest rank's time.  Checked
here with two gloo ranks on the CPU (127.0.0.1 rendezvous)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [10.0, 25.0][rank]
    units_local = [1000.0, 3000.0][rank]
    ms_max, units, per_ms = bench.aggregate(ms_local, units_local, dist)
    out[rank] = (ms_max, units, per_ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_gloo():
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
    for r in range(2):
        ms_max, units, per_ms = out[r]
        assert ms_max == 25.0 and units == 4000.0 and per_ms == pytest.approx(160.0)


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(4.0, 100.0) == (4.0, 100.0, 25.0)

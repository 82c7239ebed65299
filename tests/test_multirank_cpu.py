"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with its own
time and units; the whole-job number takes the slowest rank and all units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [100.0, 250.0][rank]                 # rank 1 is the slow one
    ms, units, value = bench.aggregate(ms_local, 1000.0 * (rank + 1), dist, "cpu")
    out[rank] = (ms, units, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_max_time_and_all_units():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, units, value = out[r]
        assert ms == 250.0 and units == 3000.0
        assert value == pytest.approx(3000.0 / 0.25)


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(200.0, 500.0) == (200.0, 500.0, 2500.0)

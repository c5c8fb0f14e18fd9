"""The multi-GPU form of the benchmark is replicas only: every rank solves its
own copy of the workload, and the job value is the units of all ranks over the
slowest rank's time.  That aggregation runs here on world_size 2 over gloo."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = 100.0                      # per rank (weak scaling)
    seconds = 1.0 + rank               # the slowest rank takes 2 s
    value, tmax = bench.replica_value(units, seconds, world, device="cpu")
    out[rank] = (value, tmax)
    dist.destroy_process_group()


def test_replica_value_uses_max_time_over_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, tmax = out[r]
        assert tmax == pytest.approx(2.0)
        assert value == pytest.approx(2 * 100.0 / 2.0)

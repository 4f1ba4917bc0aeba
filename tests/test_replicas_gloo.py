"""Multi-GPU runs are independent replicas (the solves exchange no data):
the benchmark's aggregation -- barrier, slowest rank's time, summed work --
checked with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as td
    import bench
    td.init_process_group("gloo", rank=rank, world_size=world)
    td.barrier()
    t, c = bench.aggregate(td, 10.0 * (rank + 1), 100 * (rank + 1), "cpu")
    q.put((rank, t, c))
    td.destroy_process_group()


def test_replica_aggregation_world2_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, c in out:
        assert t == 20.0 and c == 300.0
